// Host check of the persistent row-streaming kernels' work plan (compiled by
// tests/test_tc_layout.py with a plain C++ compiler).  For many image
// shapes and CTA counts, every item is decoded the way the convolution and
// weight-gradient kernels decode it (band fastest, then row block, then
// image), and every (image, row, column band) must be covered by exactly
// one item, every item taken by exactly one CTA (b, b + grid, ...), the grid
// must fit the slots, and the items must fit one pass whenever rc could
// still grow.
#define __host__
#define __device__
#include <cstdio>
#include <vector>

#include "../paper_1705_00614_gb300/csrc/swe_conv_tc.cuh"

using namespace swe;

static int fails = 0;

static void check(int n, int h, int w, int slots) {
    const RowPlan p = row_plan(n, h, w, slots);
    const int tpr = (w + TCM - 1) / TCM;
    bool bad = p.rc < 1 || p.rc > h || (h >= 4 && p.rc < 4) || p.grid < 1 || p.grid > slots ||
               p.grid > p.nitems || (p.rc < h && p.nitems > slots);
    const int rcn = (h + p.rc - 1) / p.rc;
    if (p.nitems != n * tpr * rcn) bad = true;
    std::vector<int> hit((size_t)n * h * tpr, 0), taken(p.nitems, 0);
    for (int b = 0; b < p.grid; ++b)
        for (int item = b; item < p.nitems; item += p.grid) {
            ++taken[item];
            const int jt = item % tpr, ri = (item / tpr) % rcn, img = item / (tpr * rcn);
            const int r0 = ri * p.rc, nt = (p.rc < h - r0 ? p.rc : h - r0);
            if (img >= n || nt < 1) {
                bad = true;
                continue;
            }
            for (int r = r0; r < r0 + nt; ++r) ++hit[((size_t)img * h + r) * tpr + jt];
        }
    for (int t : taken)
        if (t != 1) bad = true;
    for (int c : hit)
        if (c != 1) bad = true;
    if (bad && fails++ < 5) std::printf("n=%d h=%d w=%d slots=%d: rc=%d items=%d grid=%d\n", n, h, w, slots, p.rc, p.nitems, p.grid);
}

int main() {
    const int ws[] = {16, 48, 112, 128, 129, 130, 256, 300, 1024, 2048, 4096, 15360};
    const int slots[] = {1, 2, 7, 152, 456};
    int cases = 0;
    for (int n = 1; n <= 4; ++n)
        for (int h = 1; h <= 96; ++h)
            for (int w : ws)
                for (int s : slots) {
                    check(n, h, w, s);
                    ++cases;
                }
    for (int h : {256, 512, 1024, 2048, 4096})
        for (int s : slots) {
            check(1, h, h, s);
            ++cases;
        }
    std::printf("%d plans checked\n", cases);
    std::printf(fails ? "FAIL %d\n" : "ok\n", fails);
    return fails ? 1 : 0;
}
