// Learned sub-grid closure for the 4x coarser level of the hierarchical grid
// system (Sec. 2.2, Fig. 1): a 4-layer 3x3 convolutional network
// (5 -> 32 -> 32 -> 32 -> 3 channels, ReLU between layers) that maps the
// coarse state (H, Ux, Uy, b, n_M) to corrections of the coarse cells' net
// face-flux sums (the Fh, Fv that the final update K8 applies).
//
// Tensor-core kernels: BF16 operands, FP32 accumulation, NHWC activations.
// Forward and data-gradient convolutions are implicit GEMMs over (pixel) x
// (tap, input channel) on the fifth-generation tensor cores (tcgen05.mma,
// accumulator in tensor memory); the weight gradient is, per tap, a GEMM
// of (output channel) x (input channel) over pixels on the same tensor
// cores, reduced over CTAs in a fixed order.  Channel counts are padded: inputs to multiples of
// 16 (the MMA K step), outputs to 16 or 32 (the MMA N).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/swe.h"
#include "swe_conv_tc.cuh"
#include "swe_launch.h"
#include "swe_ptx.cuh"

using namespace swe;

namespace {

int cfail(int code, const std::string& m) {
    set_last_error(m.c_str());
    return code;
}

#define CKC(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return cfail(SWE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

constexpr int TY = 8, TX = 16;   // the image height and width are multiples of these
constexpr int NLAYER = 4;
constexpr int CH[NLAYER + 1] = {5, 32, 32, 32, 3};
constexpr int CIP[NLAYER] = {16, 32, 32, 32};  // padded input channels
constexpr int COP[NLAYER] = {32, 32, 32, 16};  // padded output channels

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Output handling of the convolution kernel.
enum ConvMode {
    MODE_RELU_BF16 = 0,    // + bias, ReLU, BF16 output (hidden layers)
    MODE_LINEAR_F32 = 1,   // + bias, FP32 output (last layer)
    MODE_MASK_BF16 = 2,    // no bias; output x (mask > 0), BF16 (data gradient through a ReLU)
};

// y[n, i, j, o] = sum_{tap, c} x[n, i+dy-1, j+dx-1, c] * W[tap][o][c] (+ bias)
// x: BF16 [N][H][W][CI] (through the TMA map xmap); W: BF16 [9][CO][CI].
//
// Fifth-generation tensor cores.  A persistent CTA of 4 warps keeps all nine
// taps' weights in shared memory and takes work items of up to `rc` rows of
// one 128-pixel column band.  One thread streams the input rows (TMA boxes
// of 8 channels x 130 pixels, zero outside the image) into a ring of TC_RS
// row slots, four rows ahead, and issues for each tile (one output row of
// the band) 9 * CI / 16 MMAs (M = 128 pixels, N = CO, K = 16 channels; tap
// (dy, dx) reads the slot of input row i + dy - 1 started dx pixels later)
// into one of two tensor-memory accumulators, committed to that
// accumulator's mbarrier.  The next tile's MMAs are issued before the warps
// read the current tile's accumulators back (tcgen05.ld) for the epilogue;
// a CTA barrier per tile frees the other accumulator and the oldest slot.
// Waits are bounded: on a timeout *err is set, the CTA waits (bounded) for
// the copies and MMAs it issued, frees its tensor memory and stops.
template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(128) k_conv(const __grid_constant__ CUtensorMap xmap, const __nv_bfloat16* __restrict__ w,
                                              const float* __restrict__ bias, void* __restrict__ out,
                                              const __nv_bfloat16* __restrict__ mask, int N, int H, int W,
                                              int CO_STORE, int rc, int nitems, unsigned* __restrict__ err) {
    constexpr int NKC = CI / 8;
    static_assert(CO == 16 || CO == 32, "MMA N");
    // row ring, then the weights (dynamic shared memory, 128-byte aligned)
    extern __shared__ __align__(128) unsigned char csm[];
    unsigned char* const sA = csm + ((128u - (smem_u32(csm) & 127u)) & 127u);
    unsigned char* const sW = sA + conv_a_bytes<CI>();
    __shared__ __align__(8) unsigned long long full[TC_RS];
    __shared__ __align__(8) unsigned long long mdone[2];
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tmem_alloc(&s_taddr, 64);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < TC_RS; ++q) mbar_init(&full[q], 1);
        mbar_init(&mdone[0], 1);
        mbar_init(&mdone[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    // weights: global [tap][o][c] -> shared [tap][kc][o][8]
    for (int e = tid; e < 9 * CO * NKC; e += 128) {
        const int tap = e / (CO * NKC), o = (e / NKC) % CO, kc = e % NKC;
        *reinterpret_cast<uint4*>(&sW[conv_w_stage<CI, CO>(tap, kc, o)]) =
            *reinterpret_cast<const uint4*>(&w[((size_t)tap * CO + o) * CI + 8 * kc]);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    const uint32_t aBase = smem_u32(sA), wBase = smem_u32(sW);
    constexpr uint32_t IDESC = idesc_bf16_f32(TCM, CO);
    const int tpr = (W + TCM - 1) / TCM, rcn = (H + rc - 1) / rc;
    // rows copied and tiles issued by this CTA so far (the ring slot and the
    // mbarrier phase of a row or tile follow from its running index); thread
    // 0 also tracks how far it has waited, for the shutdown after a timeout
    uint32_t grow = 0, gtile = 0;
    uint32_t rows_issued = 0, rows_seen = 0, tiles_issued = 0;

    auto issue_row = [&](uint32_t R, int n, int gi, int j0) {
        const int slot = (int)(R % TC_RS);
        unsigned long long* bar = &full[slot];
        mbar_expect_tx(bar, (unsigned)(NKC * (TCM + 2) * 16));
#pragma unroll
        for (int kc = 0; kc < NKC; ++kc) tma_load_4d(sA + conv_a_stage<CI>(slot, kc, 0), &xmap, 8 * kc, j0 - 1, gi, n, bar);
        rows_issued = R + 1;
    };
    auto wait_row = [&](uint32_t R) {
        if (R < rows_seen) return true;
        const bool ok = mbar_wait_bounded(&full[R % TC_RS], (R / TC_RS) & 1u);
        if (ok) rows_seen = R + 1;
        return ok;
    };
    // tile G (accumulator G & 1) from the input rows R .. R + 2
    auto issue_mma = [&](uint32_t G, uint32_t R) {
        const uint32_t tacc = taddr + 32u * (G & 1u);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int slot = (int)((R + tap / 3) % TC_RS);
#pragma unroll
            for (int s = 0; s < CI / 16; ++s) {
                const uint64_t ad = smem_desc(aBase + conv_a_off<CI>(slot, tap % 3, s), TC_A_LBO, TC_SBO);
                const uint64_t bd = smem_desc(wBase + conv_b_off<CI, CO>(tap, s), conv_b_lbo<CO>(), TC_SBO);
                tc_mma_bf16(tacc, ad, bd, IDESC, (tap | s) != 0 ? 1u : 0u);
            }
        }
        tc_commit(&mdone[G & 1u]);
        tiles_issued = G + 1;
    };

    bool stop = false;
    for (int item = blockIdx.x; item < nitems && !stop; item += gridDim.x) {
        const int jt = item % tpr, rci = (item / tpr) % rcn, n = item / (tpr * rcn);
        const int r0 = rci * rc, nt = min(rc, H - r0), nr = nt + 2, j0 = jt * TCM;
        if (tid == 0) {
            fence_proxy_async();  // earlier generic accesses to the ring precede the copies
            for (int q = 0; q < 4 && q < nr; ++q) issue_row(grow + q, n, r0 - 1 + q, j0);
            if (wait_row(grow) && wait_row(grow + 1) && wait_row(grow + 2)) {
                tc_fence_after();
                issue_mma(gtile, grow);
            } else {
                s_abort = 1;
            }
        }
        for (int k = 0; k < nt; ++k) {
            if (tid == 0 && !s_abort) {
                // row k + 4 replaces the row of tile k - 2, whose MMAs ended
                // before the last barrier; tile k + 1 needs rows k + 1 .. k + 3
                if (k + 4 < nr) issue_row(grow + k + 4, n, r0 + k + 3, j0);
                if (k + 1 < nt) {
                    if (wait_row(grow + k + 3)) {
                        tc_fence_after();
                        issue_mma(gtile + k + 1, grow + k + 1);
                    } else {
                        s_abort = 1;
                    }
                }
            }
            const uint32_t G = gtile + k;
            if (!mbar_wait_bounded(&mdone[G & 1u], (G >> 1) & 1u)) s_abort = 1;
            tc_fence_after();
            float v[CO];
            const uint32_t tl = taddr + 32u * (G & 1u) + ((uint32_t)(32 * warp) << 16);
            tmem_ld16(tl, v);
            if constexpr (CO > 16) tmem_ld16(tl + 16, v + 16);
            tmem_ld_wait();
            tc_fence_before();
            const int i = r0 + k, j = j0 + 32 * warp + lane;
            if (j < W) {
                const size_t pix = ((size_t)n * H + i) * W + j;
                if (MODE == MODE_LINEAR_F32) {
                    float* y = reinterpret_cast<float*>(out);
                    for (int o = 0; o < CO_STORE; ++o) y[pix * CO_STORE + o] = v[o] + bias[o];
                } else {
                    uint32_t pk[CO / 2];
                    if (MODE == MODE_MASK_BF16) {
                        uint32_t mk[CO / 2];
#pragma unroll
                        for (int q = 0; q < CO / 8; ++q) {
                            const uint4 m4 = *reinterpret_cast<const uint4*>(&mask[pix * CO + 8 * q]);
                            mk[4 * q] = m4.x;
                            mk[4 * q + 1] = m4.y;
                            mk[4 * q + 2] = m4.z;
                            mk[4 * q + 3] = m4.w;
                        }
#pragma unroll
                        for (int h = 0; h < CO / 2; ++h) {
                            const float m0 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(mk[h] & 0xFFFFu)));
                            const float m1 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(mk[h] >> 16)));
                            pk[h] = pack2(__float2bfloat16(m0 > 0.f ? v[2 * h] : 0.f),
                                          __float2bfloat16(m1 > 0.f ? v[2 * h + 1] : 0.f));
                        }
                    } else {
#pragma unroll
                        for (int h = 0; h < CO / 2; ++h)
                            pk[h] = pack2(__float2bfloat16(fmaxf(v[2 * h] + bias[2 * h], 0.f)),
                                          __float2bfloat16(fmaxf(v[2 * h + 1] + bias[2 * h + 1], 0.f)));
                    }
                    __nv_bfloat16* y = reinterpret_cast<__nv_bfloat16*>(out);
#pragma unroll
                    for (int q = 0; q < CO / 8; ++q)
                        *reinterpret_cast<uint4*>(&y[pix * CO + 8 * q]) =
                            make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                }
            }
            if (__syncthreads_or(s_abort)) {
                stop = true;
                break;
            }
        }
        grow += (uint32_t)nr;
        gtile += (uint32_t)nt;
    }
    if (stop && tid == 0) {
        atomicOr(err, 1u);
        // let the copies and MMAs this CTA issued finish before it leaves
        for (uint32_t R = rows_seen; R < rows_issued; ++R) mbar_wait_bounded(&full[R % TC_RS], (R / TC_RS) & 1u);
        for (uint32_t G = (tiles_issued >= 2 ? tiles_issued - 2 : 0); G < tiles_issued; ++G)
            mbar_wait_bounded(&mdone[G & 1u], (G >> 1) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, 64);
    }
}

// Weight gradient on the fifth-generation tensor cores.  For a layer with
// weights W[dy][dx][c][o] the gradient is
//   P[dy][dx][c][o] = sum over pixels p of x[p + (dy - 1, dx - 1)][c] g[p][o]
//                   = sum over pixels q of x[q + (dy - 1, 0)][c] g[q - (0, dx - 1)][o],
// one GEMM per 16-pixel K step of M = (dy, c) -- the three input rows of a
// 128-pixel row tile stacked, each row's channels followed by a chunk of
// ones (3 (CI + 8) rows, padded to 128) -- by N = (dx, o), the tile's
// output-gradient row in three copies shifted by 1 - dx pixels.  The ones
// rows give the bias gradient sum_p g[p][o].  Both operands are in the
// MN-major layout without swizzling ([chunk of 8 channels][pixel][8], 16
// bytes per pixel and chunk; K groups of 8 pixels 128 bytes apart (LBO),
// channel chunks one chunk apart (SBO)).  Input rows come straight from TMA:
// stacking dy on M needs a tile's three rows in consecutive row positions,
// so they stream through a ring of WT_RS positions followed by two shadow
// positions (second copies of the rows in positions 0 and 1) and spare
// positions that the padding rows of M read (finite data in accumulator
// rows that are never stored).  Output-gradient rows land by TMA in a raw
// ring (130 pixels from one left of the tile); warps 2 and 3 write the three
// shifted copies into the operand ring with plain shared-memory copies.
//
// A persistent CTA walks items of rows of one 128-pixel column band, keeps
// its accumulators in tensor memory and writes its partial sums once at the
// end (reduced over CTAs in a fixed order by k_wgrad_reduce).  Thread 32
// issues the copies, warps 2-3 build the shifted operands, thread 0 issues
// the MMAs; full/empty mbarriers join them (tcgen05.commit releases what
// the MMAs read).  Waits are bounded; on a timeout *err is set, every role
// waits (bounded) for what it issued, the CTA frees its tensor memory and
// writes no partials.
template <int CI, int CO>
__global__ void __launch_bounds__(128, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap gmap,
               float* __restrict__ part, float* __restrict__ bpart, int H, int W, int rc, int nitems,
               unsigned* __restrict__ err) {
    using L = WgTc<CI, CO>;
    extern __shared__ __align__(128) unsigned char wsm[];
    unsigned char* const sX = wsm + ((128u - (smem_u32(wsm) & 127u)) & 127u);
    unsigned char* const sR = sX + L::XBYTES;
    unsigned char* const sS = sR + L::RBYTES;
    __shared__ __align__(8) unsigned long long xfull[WT_RS], xempty[WT_RS];
    __shared__ __align__(8) unsigned long long rfull[WT_GR], rempty[WT_GR];
    __shared__ __align__(8) unsigned long long sfull[WT_GS], sempty[WT_GS];
    __shared__ __align__(8) unsigned long long tdone;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // zero the input ring, then ones in the last chunk of every row position
    for (uint32_t e = tid; e < L::XBYTES / 16; e += 128)
        *reinterpret_cast<uint4*>(sX + 16 * e) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const uint32_t one2 = 0x3F803F80u;  // two BF16 ones
    for (uint32_t e = tid; e < (uint32_t)L::NPOS * TC_APAD; e += 128) {
        const uint32_t pos = e / TC_APAD, px = e % TC_APAD;
        *reinterpret_cast<uint4*>(sX + wt_x_stage<CI, CO>((int)pos, L::NCX, (int)px)) = make_uint4(one2, one2, one2, one2);
    }
    if (warp == 0) {
        tmem_alloc(&s_taddr, L::TMC);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < WT_RS; ++q) {
            mbar_init(&xfull[q], 1);
            mbar_init(&xempty[q], 1);
        }
        for (int q = 0; q < WT_GR; ++q) {
            mbar_init(&rfull[q], 1);
            mbar_init(&rempty[q], WT_COPY_THREADS);
        }
        for (int q = 0; q < WT_GS; ++q) {
            mbar_init(&sfull[q], WT_COPY_THREADS);
            mbar_init(&sempty[q], 1);
        }
        mbar_init(&tdone, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    const int tpr = (W + TCM - 1) / TCM, rcn = (H + rc - 1) / rc;

    if (tid == 32) {
        // copies: per item the input rows r0 - 1 and r0, then per output row
        // k the input row r0 + k + 1 and the gradient row r0 + k (the order
        // they are consumed in); a slot is refilled once it is released
        uint32_t xR = 0, gR = 0, xlap = 0, glap = 0;
        int xs = 0, gs = 0;
        auto load_x = [&](int n, int row, int j0) {
            if (xlap > 0 && !mbar_wait_bounded(&xempty[xs], (xlap - 1) & 1u)) return false;
            constexpr unsigned bytes = (unsigned)(L::NCX * (TCM + 2) * 16);
            mbar_expect_tx(&xfull[xs], xs < 2 ? 2u * bytes : bytes);
#pragma unroll
            for (int kc = 0; kc < L::NCX; ++kc) {
                tma_load_4d(sX + wt_x_stage<CI, CO>(xs, kc, 0), &xmap, 8 * kc, j0 - 1, row, n, &xfull[xs]);
                if (xs < 2)
                    tma_load_4d(sX + wt_x_stage<CI, CO>(xs + WT_RS, kc, 0), &xmap, 8 * kc, j0 - 1, row, n, &xfull[xs]);
            }
            ++xR;
            if (++xs == WT_RS) {
                xs = 0;
                ++xlap;
            }
            return true;
        };
        auto load_g = [&](int n, int row, int j0) {
            if (glap > 0 && !mbar_wait_bounded(&rempty[gs], (glap - 1) & 1u)) return false;
            mbar_expect_tx(&rfull[gs], (unsigned)(L::NCG * (TCM + 2) * 16));
#pragma unroll
            for (int kc = 0; kc < L::NCG; ++kc)
                tma_load_4d(sR + wt_raw_stage<CI, CO>(gs, kc, 0), &gmap, 8 * kc, j0 - 1, row, n, &rfull[gs]);
            ++gR;
            if (++gs == WT_GR) {
                gs = 0;
                ++glap;
            }
            return true;
        };
        bool ok = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int jt = item % tpr, ri = (item / tpr) % rcn, n = item / (tpr * rcn);
            const int r0 = ri * rc, nt = min(rc, H - r0), j0 = jt * TCM;
            ok = load_x(n, r0 - 1, j0) && load_x(n, r0, j0);
            for (int k = 0; k < nt && ok; ++k) ok = load_x(n, r0 + k + 1, j0) && load_g(n, r0 + k, j0);
        }
        if (!ok) {
            atomicOr(err, 1u);
            atomicOr(&s_abort, 1);
        }
        // copies in flight (the newest row of each slot) land before the CTA exits
        for (uint32_t R = xR > WT_RS ? xR - WT_RS : 0; R < xR; ++R)
            mbar_wait_bounded(&xfull[R % WT_RS], (R / WT_RS) & 1u);
        for (uint32_t R = gR > WT_GR ? gR - WT_GR : 0; R < gR; ++R)
            mbar_wait_bounded(&rfull[R % WT_GR], (R / WT_GR) & 1u);
    } else if (warp >= 2) {
        // shifted operands (warps 2 and 3): copy dx of gradient row R holds
        // raw pixels 2 - dx .. 129 - dx (the raw row starts one pixel left of
        // the tile)
        static_assert(WT_COPY_THREADS == 64, "warps 0 and 1 issue the MMAs and the copies");
        const int ct = tid - (128 - WT_COPY_THREADS);
        uint32_t R = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int ri = (item / tpr) % rcn, nt = min(rc, H - ri * rc);
            for (int k = 0; k < nt; ++k, ++R) {
                const uint32_t rs = R % WT_GR, ss = R % WT_GS;
                if (!mbar_wait_bounded(&rfull[rs], (R / WT_GR) & 1u) ||
                    (R >= WT_GS && !mbar_wait_bounded(&sempty[ss], ((R / WT_GS) - 1) & 1u))) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int i = 0; i < L::CPY; ++i) {
                    int dx, oc, p;
                    wt_copy_index<CI, CO>(ct + WT_COPY_THREADS * i, dx, oc, p);
                    *reinterpret_cast<uint4*>(sS + wt_s_stage<CI, CO>((int)ss, dx, oc, p)) =
                        *reinterpret_cast<const uint4*>(sR + wt_raw_stage<CI, CO>((int)rs, oc, wt_copy_src(dx, p)));
                }
                fence_proxy_async();  // the stores precede the MMAs' reads
                mbar_arrive(&rempty[rs]);
                mbar_arrive(&sfull[ss]);
            }
        }
        if (!ok) {
            atomicOr(err, 1u);
            atomicOr(&s_abort, 1);
        }
    } else if (tid == 0) {
        // MMAs: one per 16-pixel K step, M = the stacked input rows (read
        // from pixel 1 of the row positions: the tile's own pixels), N = the
        // three shifted gradient copies
        const uint32_t xbase = smem_u32(sX), sbase = smem_u32(sS);
        constexpr uint32_t IDESC = wt_idesc<CO>();
        uint32_t x_seen = 0, cx = 0, R = 0;
        bool ok = true, first = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int ri = (item / tpr) % rcn, nt = min(rc, H - ri * rc);
            for (int k = 0; k < nt; ++k, ++R) {
                while (x_seen <= cx + k + 2) {
                    if (!mbar_wait_bounded(&xfull[x_seen % WT_RS], (x_seen / WT_RS) & 1u)) {
                        ok = false;
                        break;
                    }
                    ++x_seen;
                }
                const uint32_t ss = R % WT_GS;
                if (!ok || !mbar_wait_bounded(&sfull[ss], (R / WT_GS) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t xsl = (cx + k) % WT_RS;
                const uint64_t ad = wt_a_desc<CI, CO>(xbase, (int)xsl);
                const uint64_t bd = wt_b_desc<CI, CO>(sbase, (int)ss);
#pragma unroll
                for (int s = 0; s < TCM / 16; ++s)
                    tc_mma_bf16(taddr, ad + wt_kstep(s), bd + wt_kstep(s), IDESC, (first && s == 0) ? 0u : 1u);
                first = false;
                // this tile is the last reader of its gradient copies and of
                // input row k (and, at the item's end, of input rows k + 1, k + 2)
                tc_commit(&sempty[ss]);
                tc_commit(&xempty[xsl]);
                if (k == nt - 1) {
                    tc_commit(&xempty[(xsl + 1) % WT_RS]);
                    tc_commit(&xempty[(xsl + 2) % WT_RS]);
                }
            }
            cx += (uint32_t)(nt + 2);
        }
        tc_commit(&tdone);
        if (!mbar_wait_bounded(&tdone, 0u)) ok = false;
        if (!ok) {
            atomicOr(err, 1u);
            atomicOr(&s_abort, 1);
        }
        if (first) atomicOr(&s_abort, 2);  // no tile: the partials are zero
    }
    tc_fence_before();
    __syncthreads();
    __syncwarp();
    tc_fence_after();
    const int ab = s_abort;
    if (!(ab & 1)) {
        // accumulator row m sits in lane m: chunk m / 8 of the stacked rows;
        // column dx * CO + o
        const int m = 32 * warp + lane;
        int dy, kc;
        wt_row<CI, CO>(m, dy, kc);
        const int c = 8 * kc + (m & 7);
        const bool wrow = dy < 3 && kc < L::NCX;
        const bool brow = m == 8 * L::NCX;  // first ones row (dy = 0)
        float* P = part + (size_t)blockIdx.x * 9 * CI * CO;
        float v[16];
#pragma unroll
        for (int col = 0; col < L::N; col += 16) {
            tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)col, v);
            tmem_ld_wait();
            if (ab & 2) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
            const int dx = col / CO, o0 = col % CO;
            if (wrow) {
                float4* dst = reinterpret_cast<float4*>(P + ((size_t)(3 * dy + dx) * CI + c) * CO + o0);
#pragma unroll
                for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
            if (brow && dx == 1) {
#pragma unroll
                for (int i = 0; i < 16; ++i) bpart[(size_t)blockIdx.x * CO + o0 + i] = v[i];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, L::TMC);
    }
}

// Fixed-order sum of the per-CTA partials -> FP32 gradients in the master
// layout [3][3][ci][co] (real channels) and [co].  One CTA per 32 outputs
// (lane = output): warp k sums the partials k, k + 8, k + 16, ... in order,
// then the 8 warp sums are added in warp order.
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float* __restrict__ part, const float* __restrict__ bpart,
                                                      int nblk, int CIp, int COp, int ci, int co,
                                                      float* __restrict__ gw, float* __restrict__ gb) {
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    const int nw = 9 * ci * co;
    float s = 0.f;
    if (e < nw) {
        const int tap = e / (ci * co), c = (e / co) % ci, o = e % co;
        const size_t off = (size_t)tap * CIp * COp + (size_t)c * COp + o;
        for (int b = warp; b < nblk; b += 8) s += part[(size_t)b * 9 * CIp * COp + off];
    } else if (e < nw + co) {
        const int o = e - nw;
        for (int b = warp; b < nblk; b += 8) s += bpart[(size_t)b * COp + o];
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += red[k][lane];
        if (e < nw) gw[e] = t;
        else if (e < nw + co) gb[e - nw] = t;
    }
}

// Master FP32 weights [3][3][ci][co] -> BF16 kernel layout [9][COp][CIp]
// (zero padded).  flip != 0 gives the data-gradient weights: W'[tap][c][o]
// = W[8 - tap][o][c] (taps reversed, channels swapped).
__global__ void k_pack_w(const float* __restrict__ wm, __nv_bfloat16* __restrict__ wk, int ci, int co, int CIp, int COp,
                         int flip) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (!flip) {
        if (e >= 9 * COp * CIp) return;
        const int tap = e / (COp * CIp), o = (e / CIp) % COp, c = e % CIp;
        const float v = (o < co && c < ci) ? wm[(size_t)tap * ci * co + (size_t)c * co + o] : 0.f;
        wk[e] = __float2bfloat16(v);
    } else {
        // output channels of the gradient conv are the layer's inputs (CIp)
        if (e >= 9 * CIp * COp) return;
        const int tap = e / (CIp * COp), c = (e / COp) % CIp, o = e % COp;
        const float v = (o < co && c < ci) ? wm[(size_t)(8 - tap) * ci * co + (size_t)c * co + o] : 0.f;
        wk[e] = __float2bfloat16(v);
    }
}

// Mean-squared error over the real output channels and its gradient, as
// BF16 [N][H][W][16] (channels 3.. zero) for the last layer's backward pass.
// A warp's 32 pixels are summed in FP32 (fixed shuffle tree) and the block's
// warps in FP64: one FP64 operation per warp rather than several per pixel.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, __nv_bfloat16* __restrict__ gy,
                      double* __restrict__ part, long long npix, int co, float scale) {
    __shared__ double red[8];
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (p < npix) {
        __nv_bfloat16 gv[16];
        for (int o = 0; o < 16; ++o) {
            float g = 0.f;
            if (o < co) {
                const float d = y[p * co + o] - t[p * co + o];
                l = fmaf(d, d, l);
                g = 2.f * d * scale;
            }
            gv[o] = __float2bfloat16(g);
        }
        uint4* dst = reinterpret_cast<uint4*>(&gy[p * 16]);
        dst[0] = *reinterpret_cast<const uint4*>(&gv[0]);
        dst[1] = *reinterpret_cast<const uint4*>(&gv[8]);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += red[i];
        part[blockIdx.x] = s;
    }
}

// Fixed-order sum of n values by one CTA of 256 threads (strided partial
// sums, then a fixed tree).
__global__ void k_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Adam (Kingma & Ba 2015) on all parameters, FP32.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Corrections apply to interior wet cells only: the cell and its four
// neighbours wet, and at least CORR_HMIN deep.  At shorelines the coarse
// and fine wet areas differ by whole sub-cells, which no flux correction of
// the coarse cell can represent.
constexpr float CORR_HMIN = 0.05f;
// Standardised network inputs and outputs are clipped to +-CLIP.
constexpr float CLIP = 10.f;

template <class T>
__device__ __forceinline__ bool corr_cell(const Grid<T>& g, int buf, size_t k, T eps) {
    const T* H = g.H[buf];
    const size_t p = (size_t)g.pitch;
    return (float)H[k] >= CORR_HMIN && is_wet(H[k], g.b[k], eps) && is_wet(H[k - 1], g.b[k - 1], eps) &&
           is_wet(H[k + 1], g.b[k + 1], eps) && is_wet(H[k - p], g.b[k - p], eps) && is_wet(H[k + p], g.b[k + p], eps);
}

// Coarse-grid input features: (H, Ux, Uy, b, n) of the state at the
// control block's step parity, standardised per channel and clipped,
// BF16 [ny][nx][16].
template <class T>
__global__ void k_features(const Grid<T> g, const Ctl* __restrict__ ctl, T eps, const float* __restrict__ nrm,
                           __nv_bfloat16* __restrict__ xf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= g.nx) return;
    const int buf = (int)(ctl->step & 1);
    const size_t k = (size_t)(j + PAD) * g.pitch + (i + PAD);
    const T h = g.H[buf][k], bb = g.b[k];
    const bool wet = is_wet(h, bb, eps);
    const bool wall = !(bb < T(WALL_TEST));
    const float v[5] = {(float)h, wet ? (float)(g.Qx[buf][k] / h) : 0.f, wet ? (float)(g.Qy[buf][k] / h) : 0.f,
                        wall ? 0.f : (float)bb, (float)g.n[k]};
    __nv_bfloat16* o = &xf[((size_t)j * g.nx + i) * 16];
#pragma unroll
    for (int c = 0; c < 16; ++c)
        o[c] = __float2bfloat16(c < 5 ? fminf(CLIP, fmaxf(-CLIP, (v[c] - nrm[c]) / nrm[5 + c])) : 0.f);
}

// CNN output -> corrections of interior wet cells (pass 0: write, sum the
// depth correction; pass 1: subtract its mean over those cells, so the
// corrections add no mass).
template <class T>
__global__ void k_corrections(const Grid<T> g, const Ctl* __restrict__ ctl, T eps, const float* __restrict__ y,
                              const float* __restrict__ nrm, T* __restrict__ corr, size_t plane,
                              double* __restrict__ acc, int pass) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    double s = 0.0, cnt = 0.0;
    if (i < g.nx) {
        const int buf = (int)(ctl->step & 1);
        const size_t k = (size_t)(j + PAD) * g.pitch + (i + PAD);
        const bool on = corr_cell(g, buf, k, eps);
        if (pass == 0) {
            const float* yy = &y[((size_t)j * g.nx + i) * 3];
            auto val = [&](int q) { return fminf(CLIP, fmaxf(-CLIP, yy[q])) * nrm[3 + q] + nrm[q]; };
            const T c0 = on ? (T)val(0) : T(0);
            corr[k] = c0;
            corr[plane + k] = on ? (T)val(1) : T(0);
            corr[2 * plane + k] = on ? (T)val(2) : T(0);
            if (on) {
                s = (double)c0;
                cnt = 1.0;
            }
        } else if (on) {
            corr[k] = (T)((double)corr[k] - acc[0] / fmax(acc[1], 1.0));
        }
    }
    if (pass == 0) {
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_down_sync(0xffffffffu, s, o);
            cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        }
        if ((threadIdx.x & 31) == 0 && cnt > 0.0) {
            atomicAdd(&acc[0], s);
            atomicAdd(&acc[1], cnt);
        }
    }
}

template <class T>
__global__ void k_restrict(const Grid<T> f, const Ctl* __restrict__ fctl, const Grid<T> c, Ctl* __restrict__ cctl) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
    const int fb = (int)(fctl->step & 1);
    if (I < c.nx) {
        double sh = 0.0, sx = 0.0, sy = 0.0;
        for (int dj = 0; dj < 4; ++dj)
            for (int di = 0; di < 4; ++di) {
                const size_t k = (size_t)(4 * J + dj + PAD) * f.pitch + (4 * I + di + PAD);
                sh += (double)f.H[fb][k];
                sx += (double)f.Qx[fb][k];
                sy += (double)f.Qy[fb][k];
            }
        const size_t kc = (size_t)(J + PAD) * c.pitch + (I + PAD);
        c.H[0][kc] = (T)(sh / 16.0);
        c.Qx[0][kc] = (T)(sx / 16.0);
        c.Qy[0][kc] = (T)(sy / 16.0);
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        const double t = fctl->t;
        memset(cctl, 0, sizeof(Ctl));
        cctl->t = t;
    }
}

// Training targets: the flux-sum corrections that turn the coarse step
// into the restricted fine state, standardised; zero correction outside the
// cells the closure acts on (decided on the state before the step).
template <class T>
__global__ void k_targets(const Grid<T> p, const Ctl* __restrict__ pctl, const Grid<T> r, const Ctl* __restrict__ rctl,
                          double h, T eps, const float* __restrict__ nrm, float* __restrict__ t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= p.nx) return;
    const int pb = (int)(pctl->step & 1), rb = (int)(rctl->step & 1);
    const double s = h / pctl->tau_last;
    const size_t k = (size_t)(j + PAD) * p.pitch + (i + PAD);
    const bool on = corr_cell(p, pb ^ 1, k, eps);
    const double d[3] = {((double)r.H[rb][k] - (double)p.H[pb][k]) * s, ((double)r.Qx[rb][k] - (double)p.Qx[pb][k]) * s,
                         ((double)r.Qy[rb][k] - (double)p.Qy[pb][k]) * s};
    float* o = &t[((size_t)j * p.nx + i) * 3];
#pragma unroll
    for (int q = 0; q < 3; ++q) o[q] = (float)(((on ? d[q] : 0.0) - nrm[q]) / nrm[3 + q]);
}

}  // namespace

namespace swe {

template <class T>
cudaError_t launch_features(const Grid<T>& g, const Ctl* ctl, T eps, const float* norm, void* x, cudaStream_t st) {
    k_features<T><<<dim3((g.nx + 127) / 128, g.ny), 128, 0, st>>>(g, ctl, eps, norm, (__nv_bfloat16*)x);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_corrections(const Grid<T>& g, const Ctl* ctl, T eps, const float* y, const float* norm, T* corr,
                               size_t plane, double* acc, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.nx + 127) / 128, g.ny);
    k_corrections<T><<<grid, 128, 0, st>>>(g, ctl, eps, y, norm, corr, plane, acc, 0);
    k_corrections<T><<<grid, 128, 0, st>>>(g, ctl, eps, y, norm, corr, plane, acc, 1);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_restrict(const Grid<T>& fine, const Ctl* fctl, const Grid<T>& coarse, Ctl* cctl, cudaStream_t st) {
    k_restrict<T><<<dim3((coarse.nx + 127) / 128, coarse.ny), 128, 0, st>>>(fine, fctl, coarse, cctl);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_targets(const Grid<T>& pred, const Ctl* pctl, const Grid<T>& ref, const Ctl* rctl, double h,
                           double eps, const float* norm, float* t, cudaStream_t st) {
    k_targets<T><<<dim3((pred.nx + 127) / 128, pred.ny), 128, 0, st>>>(pred, pctl, ref, rctl, h, T(eps), norm, t);
    return cudaGetLastError();
}

#define SWE_CLOSURE_INSTANTIATE(T)                                                                            \
    template cudaError_t launch_features<T>(const Grid<T>&, const Ctl*, T, const float*, void*, cudaStream_t);  \
    template cudaError_t launch_corrections<T>(const Grid<T>&, const Ctl*, T, const float*, const float*, T*,    \
                                               size_t, double*, cudaStream_t);                                 \
    template cudaError_t launch_restrict<T>(const Grid<T>&, const Ctl*, const Grid<T>&, Ctl*, cudaStream_t);      \
    template cudaError_t launch_targets<T>(const Grid<T>&, const Ctl*, const Grid<T>&, const Ctl*, double,        \
                                           double, const float*, float*, cudaStream_t);
SWE_CLOSURE_INSTANTIATE(float)
SWE_CLOSURE_INSTANTIATE(double)

}  // namespace swe

// --------------------------------------------------------------------- C ABI

struct swe_cnn {
    int n = 0, h = 0, w = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int nparam = 0;
    float* p = nullptr;   // master FP32 parameters, flat (w0, b0, w1, b1, ...)
    float* g = nullptr;   // gradients, same layout
    float* m = nullptr;   // Adam moments
    float* v = nullptr;
    int adam_t = 0;
    __nv_bfloat16* wk[NLAYER] = {};   // forward weights, kernel layout
    __nv_bfloat16* wd[NLAYER] = {};   // data-gradient weights
    __nv_bfloat16* act[NLAYER] = {};  // act[0] unused (input given); act[l] = output of layer l-1 (BF16)
    float* yout = nullptr;            // last layer output FP32 [n][h][w][3]
    __nv_bfloat16* gbuf[2] = {};      // gradient ping-pong, BF16 [n][h][w][32]
    int nwg = 0;                      // weight-gradient CTAs the partial buffers hold
    int ntc = 0;                      // persistent convolution CTAs
    float* part = nullptr;            // weight-gradient partials, one set per such CTA
    float* bpart = nullptr;
    double* lpart = nullptr;
    double* dloss = nullptr;
    unsigned* derr = nullptr;         // device error word (bounded waits that gave up)
    int off_w[NLAYER], off_b[NLAYER];
};

namespace {

// Synchronise the network's stream and report a device wait that gave up.
int sync_check(swe_cnn* c) {
    unsigned e = 0;
    CKC(cudaMemcpyAsync(&e, c->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
    CKC(cudaStreamSynchronize(c->st));
    if (e) return cfail(SWE_ERR_DEVICE_TIMEOUT, "a tensor-core wait timed out");
    return SWE_OK;
}

template <int CI, int CO>
constexpr size_t conv_smem_bytes() {
    return (size_t)conv_a_bytes<CI>() + conv_w_bytes<CI, CO>() + 128;  // + alignment slack
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// TMA map of a BF16 NHWC image batch [n][h][w][ci]: boxes of 8 channels x
// (TCM + 2) pixels of one row; reads outside the image return zeros.
int x_map(CUtensorMap* m, const void* x, int n, int h, int w, int ci, int box_w = TCM + 2) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cfail(SWE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[4] = {(cuuint64_t)ci, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)ci * 2, (cuuint64_t)w * ci * 2, (cuuint64_t)h * w * ci * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)box_w, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cfail(SWE_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return SWE_OK;
}

// Convolution launch: items from row_plan (rc rows of one 128-pixel column
// band, about one item per persistent CTA).
template <int CI, int CO, int MODE>
int conv(swe_cnn* c, const void* x, const __nv_bfloat16* w, const float* bias, void* out, const __nv_bfloat16* mask,
         int co_store) {
    CUtensorMap m;
    int rc = x_map(&m, x, c->n, c->h, c->w, CI);
    if (rc) return rc;
    const RowPlan p = row_plan(c->n, c->h, c->w, c->ntc);
    k_conv<CI, CO, MODE><<<p.grid, 128, conv_smem_bytes<CI, CO>(), c->st>>>(m, w, bias, out, mask, c->n, c->h, c->w,
                                                                           co_store, p.rc, p.nitems, c->derr);
    CKC(cudaGetLastError());
    return SWE_OK;
}

template <int CI, int CO, int MODE>
cudaError_t conv_attr() {
    return cudaFuncSetAttribute(k_conv<CI, CO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)conv_smem_bytes<CI, CO>());
}

// Weight gradient of one layer on the tensor cores: one persistent CTA per
// SM, items of rows of one 128-pixel column band as for the convolution.
// Returns the number of CTAs (partial-sum sets) in *nblk.
template <int CI, int CO>
int wgrad_tc(swe_cnn* c, const void* x, const void* g, int* nblk) {
    CUtensorMap xm, gm;
    int rc = x_map(&xm, x, c->n, c->h, c->w, CI);
    if (!rc) rc = x_map(&gm, g, c->n, c->h, c->w, CO);
    if (rc) return rc;
    const RowPlan p = row_plan(c->n, c->h, c->w, c->nwg);
    k_wgrad_tc<CI, CO><<<p.grid, 128, WgTc<CI, CO>::SMEM, c->st>>>(xm, gm, c->part, c->bpart, c->h, c->w, p.rc,
                                                                   p.nitems, c->derr);
    CKC(cudaGetLastError());
    *nblk = p.grid;
    return SWE_OK;
}

template <int CI, int CO>
cudaError_t wgrad_tc_attr() {
    return cudaFuncSetAttribute(k_wgrad_tc<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)WgTc<CI, CO>::SMEM);
}

int layer_fwd(swe_cnn* c, int l, const __nv_bfloat16* x, void* out) {
    const float* bias = c->p + c->off_b[l];
    switch (l) {
        case 0: return conv<16, 32, MODE_RELU_BF16>(c, x, c->wk[0], bias, out, nullptr, 32);
        case 1: return conv<32, 32, MODE_RELU_BF16>(c, x, c->wk[1], bias, out, nullptr, 32);
        case 2: return conv<32, 32, MODE_RELU_BF16>(c, x, c->wk[2], bias, out, nullptr, 32);
        default: return conv<32, 16, MODE_LINEAR_F32>(c, x, c->wk[3], bias, out, nullptr, 3);
    }
}

// Output-gradient channels of layer l as seen by its backward kernels: the
// last layer's 3 outputs travel as 16 channels (the MMA K step).
constexpr int cog(int l) { return l == NLAYER - 1 ? 16 : COP[l]; }

int pack_weights(swe_cnn* c) {
    for (int l = 0; l < NLAYER; ++l) {
        const int nel = 9 * CIP[l] * COP[l];
        k_pack_w<<<(nel + 255) / 256, 256, 0, c->st>>>(c->p + c->off_w[l], c->wk[l], CH[l], CH[l + 1], CIP[l], COP[l], 0);
        const int neld = 9 * CIP[l] * cog(l);
        k_pack_w<<<(neld + 255) / 256, 256, 0, c->st>>>(c->p + c->off_w[l], c->wd[l], CH[l], CH[l + 1], CIP[l], cog(l), 1);
    }
    CKC(cudaGetLastError());
    return SWE_OK;
}

int forward_all(swe_cnn* c, const __nv_bfloat16* x) {
    int rc = layer_fwd(c, 0, x, c->act[1]);
    if (!rc) rc = layer_fwd(c, 1, c->act[1], c->act[2]);
    if (!rc) rc = layer_fwd(c, 2, c->act[2], c->act[3]);
    if (!rc) rc = layer_fwd(c, 3, c->act[3], c->yout);
    return rc;
}

// Loss, gradients of all layers into c->g (loss value into c->dloss).
int backward_all(swe_cnn* c, const __nv_bfloat16* x, const float* target) {
    const long long npix = (long long)c->n * c->h * c->w;
    const int nb = (int)((npix + 255) / 256);
    // gbuf[0] holds the 16-channel gradient of the last layer's output
    k_mse<<<nb, 256, 0, c->st>>>(c->yout, target, c->gbuf[0], c->lpart, npix, 3, 1.0f / (float)(npix * 3));
    k_sum<<<1, 256, 0, c->st>>>(c->lpart, nb, c->dloss);
    const __nv_bfloat16* ins[NLAYER] = {x, c->act[1], c->act[2], c->act[3]};
    int cur = 0;
    for (int l = NLAYER - 1; l >= 0; --l) {
        const __nv_bfloat16* gl = c->gbuf[cur];
        // weight gradient of layer l: inputs ins[l] (CIP), output gradient gl
        int nblk = 0, rcw = 0;
        switch (l) {
            case 0: rcw = wgrad_tc<16, 32>(c, ins[0], gl, &nblk); break;
            case 3: rcw = wgrad_tc<32, 16>(c, ins[3], gl, &nblk); break;
            default: rcw = wgrad_tc<32, 32>(c, ins[l], gl, &nblk); break;
        }
        if (rcw) return rcw;
        const int nw = 9 * CH[l] * CH[l + 1] + CH[l + 1];
        k_wgrad_reduce<<<(nw + 31) / 32, 256, 0, c->st>>>(c->part, c->bpart, nblk, CIP[l], cog(l), CH[l], CH[l + 1],
                                                           c->g + c->off_w[l], c->g + c->off_b[l]);
        if (l > 0) {
            // data gradient into layer l's input, masked by that input's ReLU
            __nv_bfloat16* go = c->gbuf[cur ^ 1];
            const int rc = l == 3 ? conv<16, 32, MODE_MASK_BF16>(c, gl, c->wd[3], nullptr, go, c->act[3], 32)
                                  : conv<32, 32, MODE_MASK_BF16>(c, gl, c->wd[l], nullptr, go, c->act[l], 32);
            if (rc) return rc;
            cur ^= 1;
        }
    }
    CKC(cudaGetLastError());
    return SWE_OK;
}

}  // namespace

int swe::cnn_forward_on(swe_cnn* c, const void* x, cudaStream_t st) {
    cudaStream_t keep = c->st;
    c->st = st;
    const int rc = forward_all(c, (const __nv_bfloat16*)x);
    c->st = keep;
    return rc;
}

const float* swe::cnn_output(const swe_cnn* c) { return c->yout; }

void swe::cnn_shape(const swe_cnn* c, int* n, int* h, int* w) {
    *n = c->n;
    *h = c->h;
    *w = c->w;
}

extern "C" {

SWE_API int swe_cnn_create(int32_t n, int32_t h, int32_t w, void* stream, swe_cnn** out) {
    if (!out || n < 1 || h < TY || w < TX || h % TY || w % TX)
        return cfail(SWE_ERR_ARG, "batch shape: n >= 1, h a multiple of 8, w a multiple of 16");
    *out = nullptr;
    swe_cnn* c = new (std::nothrow) swe_cnn();
    if (!c) return cfail(SWE_ERR_OOM, "cnn");
    c->n = n;
    c->h = h;
    c->w = w;
    if (stream) {
        c->st = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return cfail(SWE_ERR_CUDA, "stream");
        }
        c->own_stream = true;
    }
    int np = 0;
    for (int l = 0; l < NLAYER; ++l) {
        c->off_w[l] = np;
        np += 9 * CH[l] * CH[l + 1];
        c->off_b[l] = np;
        np += CH[l + 1];
    }
    c->nparam = np;
    const size_t npix = (size_t)n * h * w;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        swe_cnn_destroy(c);
        return cfail(SWE_ERR_CUDA, "device attributes");
    }
    c->nwg = nsm;  // weight-gradient CTAs: one per SM
    c->ntc = 3 * nsm;  // three 71 KB CTAs fit an SM
    if (conv_attr<16, 32, MODE_RELU_BF16>() != cudaSuccess || conv_attr<32, 32, MODE_RELU_BF16>() != cudaSuccess ||
        conv_attr<32, 16, MODE_LINEAR_F32>() != cudaSuccess || conv_attr<16, 32, MODE_MASK_BF16>() != cudaSuccess ||
        conv_attr<32, 32, MODE_MASK_BF16>() != cudaSuccess || wgrad_tc_attr<16, 32>() != cudaSuccess ||
        wgrad_tc_attr<32, 32>() != cudaSuccess || wgrad_tc_attr<32, 16>() != cudaSuccess) {
        swe_cnn_destroy(c);
        return cfail(SWE_ERR_CUDA, "convolution kernel shared-memory size");
    }
    const size_t nblk = (size_t)c->nwg;
    bool ok = cudaMalloc(&c->p, np * sizeof(float)) == cudaSuccess && cudaMalloc(&c->g, np * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&c->m, np * sizeof(float)) == cudaSuccess && cudaMalloc(&c->v, np * sizeof(float)) == cudaSuccess;
    for (int l = 0; l < NLAYER && ok; ++l) {
        ok = cudaMalloc(&c->wk[l], 9 * CIP[l] * COP[l] * sizeof(__nv_bfloat16)) == cudaSuccess &&
             cudaMalloc(&c->wd[l], 9 * CIP[l] * cog(l) * sizeof(__nv_bfloat16)) == cudaSuccess;
        if (ok && l > 0) ok = cudaMalloc(&c->act[l], npix * 32 * sizeof(__nv_bfloat16)) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&c->yout, npix * 3 * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c->gbuf[0], npix * 32 * sizeof(__nv_bfloat16)) == cudaSuccess &&
         cudaMalloc(&c->gbuf[1], npix * 32 * sizeof(__nv_bfloat16)) == cudaSuccess &&
         cudaMalloc(&c->part, nblk * 9 * 32 * 32 * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c->bpart, nblk * 32 * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c->lpart, ((npix + 255) / 256) * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&c->dloss, sizeof(double)) == cudaSuccess &&
         cudaMalloc(&c->derr, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        swe_cnn_destroy(c);
        return cfail(SWE_ERR_OOM, "cnn buffers");
    }
    cudaMemsetAsync(c->p, 0, np * sizeof(float), c->st);
    cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st);
    cudaMemsetAsync(c->m, 0, np * sizeof(float), c->st);
    cudaMemsetAsync(c->v, 0, np * sizeof(float), c->st);
    *out = c;
    return SWE_OK;
}

SWE_API int swe_cnn_num_params(const swe_cnn* c) { return c ? c->nparam : 0; }

SWE_API int swe_cnn_set_params(swe_cnn* c, const float* host) {
    if (!c || !host) return cfail(SWE_ERR_ARG, "null argument");
    CKC(cudaMemcpyAsync(c->p, host, c->nparam * sizeof(float), cudaMemcpyHostToDevice, c->st));
    CKC(cudaMemsetAsync(c->m, 0, c->nparam * sizeof(float), c->st));
    CKC(cudaMemsetAsync(c->v, 0, c->nparam * sizeof(float), c->st));
    c->adam_t = 0;
    int rc = pack_weights(c);
    if (rc) return rc;
    if (int r_ = sync_check(c)) return r_;
    return SWE_OK;
}

SWE_API int swe_cnn_get_params(swe_cnn* c, float* host) {
    if (!c || !host) return cfail(SWE_ERR_ARG, "null argument");
    CKC(cudaMemcpyAsync(host, c->p, c->nparam * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    if (int r_ = sync_check(c)) return r_;
    return SWE_OK;
}

SWE_API int swe_cnn_forward(swe_cnn* c, const void* x, float* y) {
    if (!c || !x) return cfail(SWE_ERR_ARG, "null argument");
    int rc = forward_all(c, (const __nv_bfloat16*)x);
    if (rc) return rc;
    if (y) CKC(cudaMemcpyAsync(y, c->yout, (size_t)c->n * c->h * c->w * 3 * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    return SWE_OK;
}

SWE_API int swe_cnn_gradients(swe_cnn* c, const void* x, const float* target, float* grads_host, double* loss) {
    if (!c || !x || !target) return cfail(SWE_ERR_ARG, "null argument");
    int rc = forward_all(c, (const __nv_bfloat16*)x);
    if (!rc) rc = backward_all(c, (const __nv_bfloat16*)x, target);
    if (rc) return rc;
    double l = 0.0;
    CKC(cudaMemcpyAsync(&l, c->dloss, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (grads_host) CKC(cudaMemcpyAsync(grads_host, c->g, c->nparam * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    if (int r_ = sync_check(c)) return r_;
    if (loss) *loss = l / (3.0 * c->n * c->h * c->w);
    return SWE_OK;
}

SWE_API int swe_cnn_train_step(swe_cnn* c, const void* x, const float* target, float lr, double* loss) {
    if (!c || !x || !target || !(lr > 0.f)) return cfail(SWE_ERR_ARG, "bad argument");
    int rc = forward_all(c, (const __nv_bfloat16*)x);
    if (!rc) rc = backward_all(c, (const __nv_bfloat16*)x, target);
    if (rc) return rc;
    c->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow((double)b1, c->adam_t), c2 = 1.f - (float)std::pow((double)b2, c->adam_t);
    k_adam<<<(c->nparam + 255) / 256, 256, 0, c->st>>>(c->p, c->g, c->m, c->v, c->nparam, lr, b1, b2, 1e-8f, c1, c2);
    rc = pack_weights(c);
    if (rc) return rc;
    if (loss) {
        double l = 0.0;
        CKC(cudaMemcpyAsync(&l, c->dloss, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        if (int r_ = sync_check(c)) return r_;
        *loss = l / (3.0 * c->n * c->h * c->w);
    }
    return SWE_OK;
}

SWE_API void swe_cnn_destroy(swe_cnn* c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    cudaFree(c->p);
    cudaFree(c->g);
    cudaFree(c->m);
    cudaFree(c->v);
    for (int l = 0; l < NLAYER; ++l) {
        cudaFree(c->wk[l]);
        cudaFree(c->wd[l]);
        cudaFree(c->act[l]);
    }
    cudaFree(c->yout);
    cudaFree(c->gbuf[0]);
    cudaFree(c->gbuf[1]);
    cudaFree(c->part);
    cudaFree(c->bpart);
    cudaFree(c->lpart);
    cudaFree(c->dloss);
    cudaFree(c->derr);
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
}

}  // extern "C"
