// Host check of the tensor-core weight gradient's shared-memory layout
// (compiled by tests/test_tc_layout.py with a plain C++ compiler).  One
// persistent CTA's data flow is simulated on a small ragged image with the
// kernel's own staging offsets, copy split and descriptor builders: input
// rows are staged (with zero fill outside the image) into the ring and its
// shadow positions, output-gradient rows into the raw ring, the shifted
// copies are made by the copy loop, and every MMA reads its operands through
// descriptors decoded here from the descriptor's bit layout (MN-major, no
// swizzle: element (mn, k) at start + (mn / 8) * SBO + (k / 8) * LBO +
// (k % 8) * 16 + (mn % 8) * 2).  The accumulators, read back with the
// kernel's row map, must equal the weight and bias gradients summed directly
// from their definition; every address must lie inside its buffer.
#define __host__
#define __device__
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../paper_1705_00614_gb300/csrc/swe_conv_tc.cuh"

using namespace swe;

static int fails = 0;

struct Desc {
    uint32_t start, lbo, sbo;
};

static Desc decode(uint64_t d) {
    const uint64_t known = 0x3FFFull | (0x3FFFull << 16) | (0x3FFFull << 32) | (7ull << 46) | (7ull << 49) |
                           (1ull << 52) | (7ull << 61);
    if ((d & ~known) != 0 || ((d >> 46) & 7) != 1 || ((d >> 49) & 7) != 0 || ((d >> 52) & 1) != 0 ||
        ((d >> 61) & 7) != 0) {
        std::printf("bad descriptor fields %llx\n", (unsigned long long)d);
        ++fails;
    }
    return Desc{(uint32_t)(d & 0x3FFF) << 4, (uint32_t)((d >> 16) & 0x3FFF) << 4, (uint32_t)((d >> 32) & 0x3FFF) << 4};
}

static uint32_t mn_addr(const Desc& d, int mn, int k) {
    return d.start + (uint32_t)(mn / 8) * d.sbo + (uint32_t)(k / 8) * d.lbo + (uint32_t)(k % 8) * 16 +
           (uint32_t)(mn % 8) * 2;
}

// deterministic small integers, so every sum is exact in float
static float val(uint32_t seed, int a, int b, int c) {
    uint32_t h = seed * 2654435761u ^ (uint32_t)(a * 73856093) ^ (uint32_t)(b * 19349663) ^ (uint32_t)(c * 83492791);
    h ^= h >> 13;
    h *= 0x5bd1e995u;
    h ^= h >> 15;
    return (float)((int)(h % 7u) - 3);
}

template <int CI, int CO>
static void check(int H, int W) {
    using L = WgTc<CI, CO>;
    const uint32_t xbase = 0x400, rbase = xbase + L::XBYTES, sbase = rbase + L::RBYTES;
    const uint32_t end = sbase + L::SBYTES;
    std::vector<float> sm(end / 2, 0.f);  // shared memory, one float per BF16 element
    auto x = [&](int r, int p, int c) { return (r < 0 || r >= H || p < 0 || p >= W) ? 0.f : val(1, r, p, c); };
    auto g = [&](int r, int p, int o) { return (r < 0 || r >= H || p < 0 || p >= W) ? 0.f : val(2, r, p, o); };
    auto put16 = [&](uint32_t at, const float* v, uint32_t lo, uint32_t hi) {
        if (at < lo || at + 16 > hi || at % 16) {
            if (fails++ < 5) std::printf("staging address %u outside [%u, %u)\n", at, lo, hi);
            return;
        }
        for (int e = 0; e < 8; ++e) sm[at / 2 + e] = v[e];
    };
    // ones chunk of every row position
    for (int pos = 0; pos < L::NPOS; ++pos)
        for (int p = 0; p < TC_APAD; ++p) {
            const float one[8] = {1, 1, 1, 1, 1, 1, 1, 1};
            put16(xbase + wt_x_stage<CI, CO>(pos, L::NCX, p), one, xbase, rbase);
        }
    // each (dx, chunk, pixel) of a shifted row is written exactly once
    {
        std::vector<int> hit(3 * L::NCG * TCM, 0);
        for (int ct = 0; ct < WT_COPY_THREADS; ++ct)
            for (int i = 0; i < L::CPY; ++i) {
                int dx, oc, p;
                wt_copy_index<CI, CO>(ct + WT_COPY_THREADS * i, dx, oc, p);
                if (dx < 0 || dx > 2 || oc < 0 || oc >= L::NCG || p < 0 || p >= TCM) ++fails;
                else ++hit[(dx * L::NCG + oc) * TCM + p];
            }
        for (int h : hit)
            if (h != 1) ++fails;
    }
    std::vector<float> D((size_t)128 * L::N, 0.f);
    const int tpr = (W + TCM - 1) / TCM;
    uint32_t xR = 0, gR = 0, cx = 0;
    // one CTA, one item per 128-pixel column band over all H rows
    for (int item = 0; item < tpr; ++item) {
        const int j0 = item * TCM, nt = H;
        auto load_x = [&](int row) {
            const int slot = (int)(xR % WT_RS);
            for (int kc = 0; kc < L::NCX; ++kc)
                for (int p = 0; p < TCM + 2; ++p) {
                    float v[8];
                    for (int e = 0; e < 8; ++e) v[e] = x(row, j0 - 1 + p, 8 * kc + e);
                    put16(xbase + wt_x_stage<CI, CO>(slot, kc, p), v, xbase, rbase);
                    if (slot < 2) put16(xbase + wt_x_stage<CI, CO>(slot + WT_RS, kc, p), v, xbase, rbase);
                }
            ++xR;
        };
        load_x(-1);
        load_x(0);
        for (int k = 0; k < nt; ++k) {
            load_x(k + 1);
            // raw gradient row k, then its shifted copies
            const int rs = (int)(gR % WT_GR), ss = (int)(gR % WT_GS);
            for (int oc = 0; oc < L::NCG; ++oc)
                for (int u = 0; u < TCM + 2; ++u) {
                    float v[8];
                    for (int e = 0; e < 8; ++e) v[e] = g(k, j0 - 1 + u, 8 * oc + e);
                    put16(rbase + wt_raw_stage<CI, CO>(rs, oc, u), v, rbase, sbase);
                }
            for (int e = 0; e < 3 * L::NCG * TCM; ++e) {
                int dx, oc, p;
                wt_copy_index<CI, CO>(e, dx, oc, p);
                const int u = wt_copy_src(dx, p);
                const uint32_t from = rbase + wt_raw_stage<CI, CO>(rs, oc, u);
                if (u < 0 || u >= TCM + 2 || from < rbase || from + 16 > sbase) {
                    ++fails;
                    continue;
                }
                put16(sbase + wt_s_stage<CI, CO>(ss, dx, oc, p), &sm[from / 2], sbase, end);
            }
            ++gR;
            // the tile's MMAs
            const int xsl = (int)((cx + k) % WT_RS);
            for (int s = 0; s < TCM / 16; ++s) {
                const Desc a = decode(wt_a_desc<CI, CO>(xbase, xsl) + wt_kstep(s));
                const Desc b = decode(wt_b_desc<CI, CO>(sbase, ss) + wt_kstep(s));
                for (int m = 0; m < 128; ++m)
                    for (int kk = 0; kk < 16; ++kk) {
                        const uint32_t at = mn_addr(a, m, kk);
                        if (at < xbase || at + 2 > rbase) {
                            if (fails++ < 5) std::printf("A read %u outside the input ring (m=%d)\n", at, m);
                            continue;
                        }
                        const float av = sm[at / 2];
                        for (int n = 0; n < L::N; ++n) {
                            const uint32_t bt = mn_addr(b, n, kk);
                            if (bt < sbase || bt + 2 > end) {
                                if (fails++ < 5) std::printf("B read %u outside the shifted copies\n", bt);
                                continue;
                            }
                            D[(size_t)m * L::N + n] += av * sm[bt / 2];
                        }
                    }
            }
        }
        cx += (uint32_t)(nt + 2);
    }
    // read back as the epilogue does and compare with the definitions
    for (int m = 0; m < 128; ++m) {
        int dy, kc;
        wt_row<CI, CO>(m, dy, kc);
        const int c = 8 * kc + (m & 7);
        for (int col = 0; col < L::N; ++col) {
            const int dx = col / CO, o = col % CO;
            double want;
            if (dy < 3 && kc < L::NCX) {
                want = 0.0;
                for (int r = 0; r < H; ++r)
                    for (int p = 0; p < W; ++p) want += (double)x(r + dy - 1, p + dx - 1, c) * g(r, p, o);
            } else if (m == 8 * L::NCX && dx == 1) {
                want = 0.0;
                for (int r = 0; r < H; ++r)
                    for (int p = 0; p < W; ++p) want += g(r, p, o);
            } else {
                continue;  // padding and the other ones rows are never stored
            }
            if ((double)D[(size_t)m * L::N + col] != want) {
                if (fails++ < 5)
                    std::printf("CI=%d CO=%d m=%d col=%d: %g vs %g\n", CI, CO, m, col, (double)D[(size_t)m * L::N + col], want);
            }
        }
    }
    // instruction descriptor: F32 accumulator, BF16 operands, both MN-major, N / 8, M / 16
    const uint32_t id = wt_idesc<CO>();
    const uint32_t expect = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                            ((uint32_t)(3 * CO / 8) << 17) | (8u << 24);
    if (id != expect) {
        std::printf("bad instruction descriptor %x\n", id);
        ++fails;
    }
    if (L::SMEM > 227u * 1024u) ++fails;
    std::printf("weight gradient CI=%d CO=%d on %dx%d checked\n", CI, CO, H, W);
}

int main() {
    check<16, 32>(9, 150);
    check<32, 32>(9, 150);
    check<32, 16>(5, 300);
    std::printf(fails ? "FAIL %d\n" : "ok\n", fails);
    return fails ? 1 : 0;
}
