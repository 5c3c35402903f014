// Shared-memory layout of the tensor-core (tcgen05) 3x3 convolution and the
// matrix descriptors its MMAs use.  Host-and-device code, so the layout can
// be checked on the host (the descriptors are decoded there and every
// element they address is compared with the intended one).
//
// A tile is TCM = 128 consecutive output pixels of one image row (the MMA's
// M).  Input rows stream through a ring of TC_RS row slots; per slot, channel
// chunk kc (8 channels = 16 bytes) and pixel p (130: the tile plus one pixel
// on each side) the shared array holds 16 bytes at
// ((slot * NKC + kc) * TC_APAD + p) * 16 (one TMA box of 130 x 16 bytes per
// slot and chunk).  With no swizzling the MMA reads K-major 8 x 16-byte core
// matrices: 8 consecutive pixels of one chunk are 128 contiguous bytes (the
// stride between 8-row groups, SBO = 128), and the next chunk along K is
// TC_APAD * 16 bytes further (LBO).  The operand of tap (dy, dx) is the slot
// of input row i + dy - 1, started dx pixels later.  Weights are held as
// [tap][kc][o][8 channels]: SBO 128, LBO = CO * 16.
#pragma once

#include <stdint.h>

namespace swe {

constexpr int TCM = 128;      // output pixels per tile (MMA M)
constexpr int TC_APAD = 136;  // shared rows per (row slot, channel chunk); >= TCM + 2
constexpr int TC_RS = 6;      // row slots: 3 rows per tile, two tiles in flight, one row loading
constexpr uint32_t TC_SBO = 128;
constexpr uint32_t TC_A_LBO = TC_APAD * 16;

template <int CI>
__host__ __device__ constexpr uint32_t conv_a_bytes() {
    return (uint32_t)TC_RS * (CI / 8) * TC_APAD * 16;
}
template <int CI, int CO>
__host__ __device__ constexpr uint32_t conv_w_bytes() {
    return 9u * (CI / 8) * CO * 16;
}
// Where 16 bytes (8 channels) are staged: row slot, channel chunk kc, pixel
// p of the tile's row plus halo; weights of tap t, chunk kc, output channel o.
template <int CI>
__host__ __device__ constexpr uint32_t conv_a_stage(int slot, int kc, int p) {
    return (uint32_t)(((slot * (CI / 8) + kc) * TC_APAD + p) * 16);
}
template <int CI, int CO>
__host__ __device__ constexpr uint32_t conv_w_stage(int tap, int kc, int o) {
    return (uint32_t)(((tap * (CI / 8) + kc) * CO + o) * 16);
}
// Offset of the A operand of a tap whose input row sits in `slot`, column
// shift dx, K step s (16 channels).
template <int CI>
__host__ __device__ constexpr uint32_t conv_a_off(int slot, int dx, int s) {
    return (uint32_t)(((slot * (CI / 8) + 2 * s) * TC_APAD + dx) * 16);
}
// Offset of the B operand (weights) of tap t, K step s.
template <int CI, int CO>
__host__ __device__ constexpr uint32_t conv_b_off(int tap, int s) {
    return (uint32_t)((tap * (CI / 8) + 2 * s) * CO * 16);
}
template <int CO>
__host__ __device__ constexpr uint32_t conv_b_lbo() {
    return (uint32_t)CO * 16;
}

// Shared-memory matrix descriptor, no swizzling: 14-bit start address, the
// leading (K-direction, between 8 x 16-byte core matrices) and stride
// (M/N-direction, between 8-row groups) byte offsets, all in 16-byte units;
// bit 46 is the descriptor version of this MMA generation; base offset,
// offset mode and swizzle mode (bits 49-52, 61-63) are 0.
__host__ __device__ constexpr uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of a dense BF16 x BF16 -> FP32 MMA with both
// operands K-major: D format F32 (bits 4-5), A and B format BF16 (bits 7-9,
// 10-12), N / 8 (bits 17-22), M / 16 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Work plan of the persistent row-streaming kernels (the convolution and the
// weight gradient): an item is rc consecutive rows (the last item of an
// image may be shorter) of one 128-pixel column band of one image; items are
// numbered band-fastest, then row block, then image, and CTA b takes items
// b, b + grid, ...  rc starts at max(4, tiles / slots) and grows until the
// items fit one pass of `slots` CTAs (a few items left for a second pass
// would double the makespan) or rc reaches h.
struct RowPlan {
    int rc, nitems, grid;
};
__host__ __device__ inline RowPlan row_plan(int n, int h, int w, int slots) {
    const int tpr = (w + TCM - 1) / TCM;
    const long long tiles = (long long)n * h * tpr;
    long long rc = (tiles + slots - 1) / slots;
    rc = rc < 4 ? 4 : rc;
    rc = rc > h ? h : rc;
    while (rc < h && (long long)n * tpr * ((h + rc - 1) / rc) > slots) ++rc;
    RowPlan p;
    p.rc = (int)rc;
    p.nitems = (int)((long long)n * tpr * ((h + rc - 1) / rc));
    p.grid = p.nitems < slots ? p.nitems : slots;
    return p;
}

// ---- Weight gradient (k_wgrad_tc) ----
// Per 16-pixel K step one MMA: M = (dy, c), the three input rows of a tile
// stacked, each row's NCX channel chunks followed by a chunk of ones
// (3 (CI + 8) rows, padded to 128); N = (dx, o), three copies of the tile's
// output-gradient row shifted by 1 - dx pixels.  Both operands MN-major
// without swizzling: element (mn, k) at start + (mn / 8) * SBO + (k / 8) *
// LBO + (k % 8) * 16 + (mn % 8) * 2, LBO = 128 (8 pixels), SBO = the chunk
// stride.  Input rows: a ring of WT_RS row positions, two shadow positions
// (positions WT_RS and WT_RS + 1 hold second copies of the rows in 0 and 1)
// and spare positions for the padding rows of M; per position NCX chunks
// of TC_APAD pixels (pixel 0 is one left of the tile) and the ones chunk.
// Output-gradient rows: a raw ring of WT_GR slots (NCG chunks of TC_APAD
// pixels, pixel 0 one left of the tile) and WT_GS slots of shifted copies
// (3 NCG chunks of TCM pixels).
constexpr int WT_RS = 8;  // input row positions of the ring
constexpr int WT_GR = 4;  // raw output-gradient row slots
constexpr int WT_GS = 2;  // shifted output-gradient operand slots
constexpr int WT_COPY_THREADS = 64;  // threads that write the shifted copies

template <int CI, int CO>
struct WgTc {
    static constexpr int NCX = CI / 8, NCG = CO / 8;  // channel chunks of x and g
    static constexpr int PCH = NCX + 1;               // chunks per row position (channels, ones)
    static constexpr int MROWS = 3 * 8 * PCH;         // real rows of M
    static constexpr int NPOS = WT_RS + 2 + (16 - 3 * PCH + PCH - 1) / PCH;
    static constexpr int N = 3 * CO;                  // MMA N: (dx, o)
    static constexpr int TMC = N <= 64 ? 64 : 128;    // accumulator columns
    static constexpr uint32_t CS = TC_APAD * 16;      // chunk stride of the TMA rings
    static constexpr uint32_t CSB = TCM * 16;         // chunk stride of the shifted copies
    static constexpr uint32_t POS = PCH * CS;         // row-position stride
    static constexpr uint32_t XBYTES = (uint32_t)NPOS * POS;
    static constexpr uint32_t RSLOT = (uint32_t)NCG * CS;
    static constexpr uint32_t SSLOT = (uint32_t)(3 * NCG) * CSB;
    static constexpr uint32_t RBYTES = WT_GR * RSLOT;
    static constexpr uint32_t SBYTES = WT_GS * SSLOT;
    static constexpr uint32_t SMEM = XBYTES + RBYTES + SBYTES + 128;
    static constexpr int CPY = 3 * NCG * TCM / WT_COPY_THREADS;  // 16-byte copies per copy thread and row
    static_assert(MROWS <= 128, "M");
    static_assert(CO == 16 || CO == 32, "MMA N");
    static_assert((3 * NCG * TCM) % WT_COPY_THREADS == 0, "copy split");
};

// Byte offsets: 8 channels of input pixel p in row position pos, chunk kc
// (kc = NCX: the ones chunk); of raw gradient pixel u in slot rs, chunk oc;
// of shifted copy dx, tile pixel p in slot ss, chunk oc.
template <int CI, int CO>
__host__ __device__ constexpr uint32_t wt_x_stage(int pos, int kc, int p) {
    return (uint32_t)pos * WgTc<CI, CO>::POS + (uint32_t)kc * WgTc<CI, CO>::CS + 16u * (uint32_t)p;
}
template <int CI, int CO>
__host__ __device__ constexpr uint32_t wt_raw_stage(int rs, int oc, int u) {
    return (uint32_t)rs * WgTc<CI, CO>::RSLOT + (uint32_t)oc * WgTc<CI, CO>::CS + 16u * (uint32_t)u;
}
template <int CI, int CO>
__host__ __device__ constexpr uint32_t wt_s_stage(int ss, int dx, int oc, int p) {
    return (uint32_t)ss * WgTc<CI, CO>::SSLOT + (uint32_t)(dx * WgTc<CI, CO>::NCG + oc) * WgTc<CI, CO>::CSB +
           16u * (uint32_t)p;
}
// Copy e (0 .. 3 NCG TCM - 1) of a gradient row: shift dx, chunk oc, tile
// pixel p; it takes raw pixel p + 2 - dx (gradient pixel j0 + p + 1 - dx).
template <int CI, int CO>
__host__ __device__ constexpr void wt_copy_index(int e, int& dx, int& oc, int& p) {
    dx = e / (WgTc<CI, CO>::NCG * TCM);
    oc = (e / TCM) % WgTc<CI, CO>::NCG;
    p = e % TCM;
}
__host__ __device__ constexpr int wt_copy_src(int dx, int p) { return p + 2 - dx; }
// Descriptors of K step 0 for the tile whose first input row sits in ring
// slot `slot` (the tile's own pixels start at pixel 1), and for shifted
// slot ss; K step s adds wt_kstep(s) (256 bytes = 16 pixels).
template <int CI, int CO>
__host__ __device__ constexpr uint64_t wt_a_desc(uint32_t xbase, int slot) {
    return smem_desc(xbase + wt_x_stage<CI, CO>(slot, 0, 1), 128u, WgTc<CI, CO>::CS);
}
template <int CI, int CO>
__host__ __device__ constexpr uint64_t wt_b_desc(uint32_t sbase, int ss) {
    return smem_desc(sbase + wt_s_stage<CI, CO>(ss, 0, 0, 0), 128u, WgTc<CI, CO>::CSB);
}
__host__ __device__ constexpr uint64_t wt_kstep(int s) { return (uint64_t)(16 * s); }
// Instruction descriptor: M = 128, N = 3 CO, both operands MN-major
// (transpose bits 15 and 16).
template <int CO>
__host__ __device__ constexpr uint32_t wt_idesc() {
    return idesc_bf16_f32(128, 3 * CO) | (1u << 15) | (1u << 16);
}
// Accumulator row m: input-row offset dy and chunk kc of the stacked rows
// (kc = NCX: a ones row; dy >= 3: padding).
template <int CI, int CO>
__host__ __device__ constexpr void wt_row(int m, int& dy, int& kc) {
    dy = (m >> 3) / WgTc<CI, CO>::PCH;
    kc = (m >> 3) % WgTc<CI, CO>::PCH;
}

}  // namespace swe
