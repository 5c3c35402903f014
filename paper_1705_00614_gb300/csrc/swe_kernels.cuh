// Kernels of one CSPH-TVD time step (Sec. 2.3; paper kernels K2-K8), as
// templates over the arithmetic type.  swe_f32.cu and swe_f64.cu instantiate
// them with different floating-point flags.
//
// Two organisations of the same arithmetic (swe_math.cuh):
//  * k_fused: one launch per step.  A CTA owns a window of WIN = 128 columns
//    (one thread per column in each of two warp groups) and streams down the
//    rows of its segment.  Input rows arrive by TMA one row per copy into
//    per-field shared-memory rings; every stage keeps the few rows its
//    consumers need in rings of its own, so one pass over the rows runs the
//    whole step with no intermediate in HBM: primitives and predictor U* ->
//    particle area H* -> forces at t_{n+1/2} + corrector + sources -> MUSCL
//    slopes and face fluxes -> final update -> forces and signal speed of
//    the new state (the next step's K3; its accelerations are stored for
//    the next step's predictor).  The dependence radius of all that is 6
//    cells, so a window produces its 116 central columns and rows
//    [6, 6 + seg_h) of its 12 + seg_h rows.
//  * staged kernels: one kernel per stage with every intermediate in device
//    memory (the paper's K2-K8 split); used for stage-by-stage comparison with
//    the oracle and the per-stage time breakdown.
#pragma once

#include <float.h>
#include <algorithm>
#include <limits.h>

#include "swe_launch.h"
#include "swe_ptx.cuh"

namespace swe {

// ------------------------------------------------------------------ time step

__device__ __forceinline__ double dmin_(double a, double b) { return a < b ? a : b; }

// tau_n from the max signal speed of the state at t_n (Fig. 2, K3).
__device__ __forceinline__ double step_tau(const Ctl* ctl, const StepP& sp, int parity, bool* clamped = nullptr) {
    double smax = __longlong_as_double((long long)ctl->smax[parity]);
    double tau;
    if (sp.dt_fixed > 0.0) tau = sp.dt_fixed;
    else if (smax > 0.0) tau = dmin_(sp.dt_max, sp.cfl * sp.dx / smax);
    else tau = sp.dt_max;
    const bool cut = ctl->t_end > 0.0 && ctl->t + tau > ctl->t_end;
    if (cut) tau = ctl->t_end - ctl->t;
    if (clamped) *clamped = cut;
    return tau;
}

// t_{n+1} after a step that applied tau_applied (tau rounded to the state
// precision): t_n + tau_applied, or t_end exactly when t_end cut the step
// (in FP32 the rounded tau would otherwise land a few ulps off t_end).
// Called before ctl->t and ctl->smax[parity] change.
__device__ __forceinline__ double step_time_after(const Ctl* ctl, const StepP& sp, int parity, double tau_applied) {
    bool cut = false;
    step_tau(ctl, sp, parity, &cut);
    return cut ? ctl->t_end : ctl->t + tau_applied;
}

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ int lin_tid() { return threadIdx.x + threadIdx.y * blockDim.x; }

// Sum over an NT-thread block in a fixed order (result valid in thread 0).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = lin_tid(), w = tid >> 5, l = tid & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (tid == 0)
        for (int i = 0; i < NT / 32; ++i) r += red[i];
    return r;
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        double u = __shfl_down_sync(0xffffffffu, v, o);
        v = (u > v || u != u) ? u : v;
    }
    const int tid = lin_tid(), w = tid >> 5, l = tid & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (tid == 0)
        for (int i = 0; i < NT / 32; ++i) r = (red[i] > r || red[i] != red[i]) ? red[i] : r;
    return r;
}

// ------------------------------------------------------------------ fused kernel
//
// Skewed row pipeline.  Window row r of stage s is processed in iteration
// k = r + LAG_s.  Lags are chosen so that every stage reads only rows that
// other threads finished in earlier iterations; one CTA barrier per
// iteration then orders everything.  Two warp groups of 128 threads (one
// thread per window column each) share the work of an iteration.
//
// Stages: S0 primitives U = Q/H; S1 forces at t_n and predictor U*; S2
// particle area change and H*; S3 forces at t_{n+1/2}, corrector, sources;
// S5 MUSCL slopes along x; S4 slopes along y and the face fluxes; S6 final
// update (K8); S7 signal speed of the new state (the next step's K3).
//
// ACC = true (contexts): S7 also stores the new state's accelerations
// (a_x, a_y) in a second pair of ping-pong planes, and the next step's S1
// loads them instead of evaluating the forces again (the friction
// coefficient, local to the cell, it computes from H, U and n), so S0 and
// S1 merge.
// Groups: L = {S0+S1 (lag 0), S2 (2), S3 (4), S7 (9)}, E = {S5 (5),
// S4 (6), S6 (7)}.
// ACC = false (caller-owned planes, no acceleration storage): groups
// L = {S0 (0), S1 (2), S2 (4), S3 (6), S5 (7)}, E = {S4 (8), S6 (9),
// S7 (11)}.
// Input rows (H, Qx, Qy, b, n and, with ACC, a_x, a_y) arrive by TMA
// one row per copy, PREF rows ahead of the row S0 reads, into per-field
// row rings.  Every ring holds a power of two of rows, so a row's slot is a
// mask of its index.  The copy of row k + PREF, issued at iteration k,
// overwrites row k + PREF - R, which must have been read for the last time
// before iteration k: R >= PREF + 1 + (the field's oldest reading lag).
// With ACC the rings are sized so that three FP32 CTAs fit on an SM.

constexpr int NT = 2 * WIN;
constexpr int NBAR = 4;   // > PREF: one mbarrier per row in flight
constexpr int PREF = 2;
static_assert(RB == 1, "the fused kernel streams one row per TMA copy");

// Vector types of the cell-major stage rings: 2 and 4 fields of one cell.
template <class T>
struct Vecs;
template <>
struct Vecs<float> {
    using v2 = float2;
    using v4 = float4;
};
struct __align__(16) dvec4 {
    double x, y, z, w;
};
template <>
struct Vecs<double> {
    using v2 = double2;
    using v4 = dvec4;
};

template <bool ACC>
struct Lags {
    static constexpr int S1 = ACC ? 0 : 2, S2 = ACC ? 2 : 4, S3 = ACC ? 4 : 6, S5 = ACC ? 5 : 7, S4 = ACC ? 6 : 8,
                         S6 = ACC ? 7 : 9, S7 = ACC ? 9 : 11;
};

template <class T, bool ACC>
struct FSmem {
    // input rings (rows).  Oldest readers, ACC: H and b S3 (row r-1), Q and
    // n S3 (own row), a S0; without ACC: H and b S3 (r-1), n S3, Q S0.
    // Later stages take b from the Eulerian ring cA.
    static constexpr int RH = ACC ? 8 : 16, RQ = ACC ? 8 : 4, RB_ = ACC ? 8 : 16, RN = ACC ? 8 : 16,
                         RA = ACC ? 4 : 1;
    static_assert(RH >= PREF + 1 + Lags<ACC>::S3 + 1 && RB_ >= PREF + 1 + Lags<ACC>::S3 + 1, "H/b ring");
    static_assert(RN >= PREF + 1 + Lags<ACC>::S3 && RQ >= PREF + 1 + (ACC ? Lags<ACC>::S3 : 0), "n/Q ring");
    static_assert(!ACC || RA >= PREF + 1, "a ring");
    // stage rings (rows); pU (U at t_n, read by S1 and S3) only without ACC:
    // with ACC, S3 forms U from the Q ring itself.  The stage rings are
    // cell-major: a row holds WIN cells of 2 or 4 fields each, so one cell's
    // fields move with one 8- or 16-byte shared-memory access (a warp's
    // 16-byte accesses to 32 consecutive cells are conflict-free).
    static constexpr int DP = ACC ? 1 : 8, DA = 8, DB = 4, DC = 4, DX = 2, DF = 2, DN = 4;
    using V2 = typename Vecs<T>::v2;
    using V4 = typename Vecs<T>::v4;
    T inH[RH][WIN];
    T inQx[RQ][WIN];
    T inQy[RQ][WIN];
    T inB[RB_][WIN];
    T inN[RN][WIN];
    T inA[NACC][RA][WIN];  // a_x, a_y at t_n (ACC only)
    V2 pU[DP][WIN];        // U at t_n (without ACC)
    V2 aU[DA][WIN];        // predictor U*
    T bH[DB][WIN];         // particle depth H*
    // (x, y) pairs sit in the first or second half of a 4-vector, so they
    // load into the aligned register pairs the packed FP32 arithmetic uses
    V4 cA[DC][WIN];        // post-Lagrangian U^x, U^y, H~ and the cell's b
    V4 cB[DC][WIN];        // post-Lagrangian U~'x, U~'y, Q~x, Q~y
    V4 sX[DX][WIN];        // x slopes of H~, U^x, U~'x, U~'y (an x face needs no U^y slope)
    V4 fX[DF][WIN];        // x-face fluxes F_Qx, F_Qy, F_H (w unused)
    V4 nS[DN][WIN];        // new state Ux, Uy, H with the cell's b
    unsigned long long bar[NBAR];
    double hq[MAX_HYDRO];
    double red[NT / 32];
    double tau;
    int last;
    int witem;
    int abort;
};


template <class T, bool ACC>
size_t fused_smem_bytes_v() {
    return sizeof(FSmem<T, ACC>) + 128;
}
template <class T>
size_t fused_smem_bytes() {
    return fused_smem_bytes_v<T, true>();
}

template <class T, bool ACC>
__device__ __forceinline__ void issue_row(FSmem<T, ACC>& s, const FusedArgs<T>& a, int buf, int r0,
                                          int gx0, int gy0, unsigned cbase) {
    using S = FSmem<T, ACC>;
    unsigned long long* bar = &s.bar[(cbase + (unsigned)r0) % NBAR];
    mbar_expect_tx(bar, (ACC ? 5u + (unsigned)NACC : 5u) * WIN * sizeof(T));
    const int y = gy0 + r0;
    tma_load_2d(&s.inH[r0 & (S::RH - 1)][0], &a.tmH[buf], gx0, y, bar);
    tma_load_2d(&s.inQx[r0 & (S::RQ - 1)][0], &a.tmQx[buf], gx0, y, bar);
    tma_load_2d(&s.inQy[r0 & (S::RQ - 1)][0], &a.tmQy[buf], gx0, y, bar);
    tma_load_2d(&s.inB[r0 & (S::RB_ - 1)][0], &a.tmB, gx0, y, bar);
    tma_load_2d(&s.inN[r0 & (S::RN - 1)][0], &a.tmN, gx0, y, bar);
    if (ACC) {
#pragma unroll
        for (int q = 0; q < NACC; ++q) tma_load_2d(&s.inA[q][r0 & (S::RA - 1)][0], &a.tmA[buf][q], gx0, y, bar);
    }
}

// One work item (a window of one grid's segment): the whole step for it.
// `cbase` counts the TMA rows this CTA has waited for so far, so the
// mbarrier phases stay consistent across the items a persistent CTA runs.
// Returns false when a bounded wait gave up (the CTA must stop).
template <class T, bool ACC, bool OPEN = false>
__device__ __forceinline__ bool fused_item(FSmem<T, ACC>& s, const FusedArgs<T>& a, const int item,
                                           unsigned& cbase) {
    using LG = Lags<ACC>;
    using S = FSmem<T, ACC>;
    using V2 = typename Vecs<T>::v2;
    using V4 = typename Vecs<T>::v4;
    const int tid = threadIdx.x;
    const int c = tid & (WIN - 1);
    const bool groupL = tid < WIN;
    const int strip = item % a.ntx, seg = item / a.ntx;
    const int x0 = strip * TW, y0 = seg * a.seg_h;
    const int tw = min(TW, a.g.nx - x0), sh = min(a.seg_h, a.g.ny - y0);
    const int gx0 = PAD + x0 - HALO, gy0 = PAD + y0 - HALO;
    const int nrows = sh + 2 * HALO;
    const long long step = *(volatile const long long*)&a.ctl->step;
    const int buf = (int)(step & 1);
    const Phys<T>& P = a.P;
    const T eps = P.eps;

    if (tid == 0) s.tau = step_tau(a.ctl, a.sp, buf);
    __syncthreads();
    const double tau = s.tau;
    if (!(tau > 0.0)) return true;  // t_end reached: every CTA skips the step
    const T tauT = (T)tau;
    const T th = T(0.5) * tauT;
    const T dth = tauT / P.h;
    // Wet-block test (the paper's K1): with no wet cell and no source in the
    // window this item reads, the step maps every output cell to itself
    // with Q = 0 (no force acts, every face flux is +0), so the item is
    // written directly.  Stamps of other items of this step may be raised
    // to step + 1 concurrently, which only keeps a block active.
    bool skip = false;
    if (a.skip && a.src_off[item] == a.src_off[item + 1]) {
        const int cx0 = max(0, x0 - HALO), cx1 = min(a.g.nx - 1, x0 + tw - 1 + HALO);
        const int cy0 = max(0, y0 - HALO), cy1 = min(a.g.ny - 1, y0 + sh - 1 + HALO);
        const int bx0 = cx0 >> ACT_LX, nbx = (cx1 >> ACT_LX) - bx0 + 1;
        const int by0 = cy0 >> ACT_LY, nby = (cy1 >> ACT_LY) - by0 + 1;
        bool active = false;
        for (int i = tid; i < nbx * nby; i += NT)
            active |= __ldcg(&a.act[(size_t)(by0 + i / nbx) * a.act_nbx + bx0 + i % nbx]) >= step;
        skip = !__syncthreads_or(active);
    }
    // skipped in this step and the two before: the output buffer was written
    // two steps ago with what this step would write (H already free of -0,
    // Q = 0, a = 0), and the item's partial sums of the last step still hold
    const unsigned hprev = a.hist ? (unsigned)a.hist[item] : 0u;
    const bool still = skip && hprev == 3u;
    if (tid < a.nh) s.hq[tid] = hydro_value(a.hydro + 4 * tid, a.ctl->t + 0.5 * (double)tauT);
    if (tid == 0 && !skip) {
        fence_proxy_async();
        for (int r = 0; r < PREF && r < nrows; ++r) issue_row<T, ACC>(s, a, buf, r, gx0, gy0, cbase);
    }
    __syncthreads();

    T* const outH = a.g.H[buf ^ 1];
    T* const outQx = a.g.Qx[buf ^ 1];
    T* const outQy = a.g.Qy[buf ^ 1];
    const bool out_col = (c >= HALO) && (c < HALO + tw);

    // ring rows (stage row indices are non-negative where they are used)
    auto rH = [&](int r) -> const T* { return s.inH[r & (S::RH - 1)]; };
    auto rQx = [&](int r) -> const T* { return s.inQx[r & (S::RQ - 1)]; };
    auto rQy = [&](int r) -> const T* { return s.inQy[r & (S::RQ - 1)]; };
    auto rB = [&](int r) -> const T* { return s.inB[r & (S::RB_ - 1)]; };
    auto rN = [&](int r) -> const T* { return s.inN[r & (S::RN - 1)]; };
    auto rA = [&](int q, int r) -> const T* { return s.inA[q][r & (S::RA - 1)]; };
    auto pU = [&](int r) { return s.pU[r & (S::DP - 1)]; };
    auto aU = [&](int r) { return s.aU[r & (S::DA - 1)]; };
    auto bH = [&](int r) { return s.bH[r & (S::DB - 1)]; };
    auto cA = [&](int r) { return s.cA[r & (S::DC - 1)]; };
    auto cB = [&](int r) { return s.cB[r & (S::DC - 1)]; };
    auto sX = [&](int r) { return s.sX[r & (S::DX - 1)]; };
    auto fX = [&](int r) { return s.fX[r & (S::DF - 1)]; };
    auto nS = [&](int r) { return s.nS[r & (S::DN - 1)]; };

    // the stages' column ranges for this thread: bit i (1..5) set when
    // c is in [i, WIN-1-i], bit 6 when c is in [4, WIN-6]
    unsigned cb = 0u;
#pragma unroll
    for (int i = 1; i <= 5; ++i) cb |= (c >= i && c <= WIN - 1 - i) ? (1u << i) : 0u;
    cb |= (c >= 4 && c <= WIN - 6) ? 64u : 0u;
    int sp = a.src_off[item];
    const int se = a.src_off[item + 1];
    // without point or distributed sources H~ = H exactly: nothing to add
    const bool has_src = sp != se || P.dist;
    T syPrev[5] = {T(0), T(0), T(0), T(0), T(0)};
    T fyPrev[3] = {T(0), T(0), T(0)}, fyCur[3] = {T(0), T(0), T(0)};
    double acc_mass = 0.0, acc_src = 0.0, acc_clip = 0.0;
    // the signal-speed max in the state precision (a max is exact in any
    // precision); a thread counts at most a segment's rows of wet cells
    T vmax = T(0);
    int acc_wet = 0;
    bool bad = false;
    bool band_wet = false;  // a wet new cell in this column's current stamp band

    // S0: primitives at row k (and, with ACC, the predictor velocity from
    // the stored accelerations of the state at t_n)
    auto stage0 = [&](int k) {
        if (k >= nrows) return;
        const T H = rH(k)[c];
        const bool wet = is_wet(H, rB(k)[c], eps);
        T ux, uy;
        div2_if(wet, rQx(k)[c], rQy(k)[c], H, ux, uy);
        if (!ACC) pU(k)[c] = V2{ux, uy};
        if (ACC) {
            // FP32: every lane evaluates (a dry cell's stored accelerations
            // are 0) and keeps the value where the cell is wet; FP64 only
            // where wet.  The friction coefficient is the cell's own (Eq. 4),
            // from H, U and n.
            T usx = T(0), usy = T(0);
            if (sizeof(T) == 4 || wet) {
                const T den = T(1) + th * friction(P, H, rN(k)[c], ux, uy);
                lin_div2(ux, uy, th, rA(0, k)[c], rA(1, k)[c], den, usx, usy);
            }
            aU(k)[c] = V2{wet ? usx : T(0), wet ? usy : T(0)};
        }
    };
    // S1: forces at t_n and predictor velocity U* (without ACC)
    auto stage1 = [&](int r) {
        if (!(r >= 1 && r <= nrows - 2 && (cb & 2u))) return;
        const T *H0 = rH(r), *Hm = rH(r - 1), *Hp = rH(r + 1);
        const T *b0 = rB(r), *bm = rB(r - 1), *bp = rB(r + 1);
        const V2 *U0 = pU(r), *Um = pU(r - 1), *Up = pU(r + 1);
        const T H = H0[c], b = b0[c];
        T usx = T(0), usy = T(0);
        if (is_wet(H, b, eps)) {
            const V2 uw = U0[c - 1], ue = U0[c + 1], us = Um[c], un = Up[c], u0 = U0[c];
            Nb<T> W{H0[c - 1], b0[c - 1], uw.x, uw.y, is_wet(H0[c - 1], b0[c - 1], eps)};
            Nb<T> E{H0[c + 1], b0[c + 1], ue.x, ue.y, is_wet(H0[c + 1], b0[c + 1], eps)};
            Nb<T> S{Hm[c], bm[c], us.x, us.y, is_wet(Hm[c], bm[c], eps)};
            Nb<T> N{Hp[c], bp[c], un.x, un.y, is_wet(Hp[c], bp[c], eps)};
            T ax, ay, phi;
            forces(P, H, b, rN(r)[c], u0.x, u0.y, W, E, S, N, ax, ay, phi);
            const T den = T(1) + th * phi;
            lin_div2(u0.x, u0.y, th, ax, ay, den, usx, usy);
        }
        aU(r)[c] = V2{usx, usy};
    };
    // S2: particle area change and H*
    auto stage2 = [&](int r) {
        if (!(r >= 2 && r <= nrows - 3 && (cb & 4u))) return;
        const T H = rH(r)[c];
        const bool wet = is_wet(H, rB(r)[c], eps);
        // FP32: evaluated on every lane, kept where the cell is wet; FP64
        // only where wet
        T hw = H;
        if (sizeof(T) == 4 || wet) {
            const V2* A0 = aU(r);
            const V2 a0 = A0[c];
            const T u = a0.x, uW = A0[c - 1].x, uE = A0[c + 1].x;
            const T v = a0.y, vS = aU(r - 1)[c].y, vN = aU(r + 1)[c].y;
            T D;
            if constexpr (sizeof(T) == 4) {
                // face means of the W/S and E/N faces as (x, y) pairs
                const f2 fm = mul2(mk2(0.5f, 0.5f), add2(mk2(uW, vS), mk2(u, v)));
                const f2 fp = mul2(mk2(0.5f, 0.5f), add2(mk2(u, v), mk2(uE, vN)));
                const f2 d = sub2(fp, fm);
                D = (d.x + d.y) * P.ih;
            } else {
                const T fxm = T(0.5) * (uW + u), fxp = T(0.5) * (u + uE);
                const T fym = T(0.5) * (vS + v), fyp = T(0.5) * (v + vN);
                D = ((fxp - fxm) + (fyp - fym)) / P.h;
            }
            hw = H / tmax(T(0.5), T(1) + th * D);
        }
        bH(r)[c] = wet ? hw : H;
    };
    // S3: forces at t_{n+1/2}, corrector and sources
    auto stage3 = [&](int r) {
        if (!(r >= 3 && r <= nrows - 4 && (cb & 8u))) return;
        const T *H0 = rH(r), *Hm = rH(r - 1), *Hp = rH(r + 1);
        const T *b0 = rB(r), *bm = rB(r - 1), *bp = rB(r + 1);
        const T *B0 = bH(r), *Bm = bH(r - 1), *Bp = bH(r + 1);
        const V2 *A0 = aU(r), *Am = aU(r - 1), *Ap = aU(r + 1);
        const T H = H0[c], b = b0[c];
        const bool wet = is_wet(H, b, eps);
        T ux, uy;
        if (ACC) {
            div2_if(wet, rQx(r)[c], rQy(r)[c], H, ux, uy);
        } else {
            const V2 u0 = pU(r)[c];
            ux = u0.x;
            uy = u0.y;
        }
        const T nm = rN(r)[c];
        T utx = T(0), uty = T(0);
        if (wet) {
            const V2 aw = A0[c - 1], ae = A0[c + 1], as = Am[c], an = Ap[c], a0 = A0[c];
            Nb<T> W{B0[c - 1], b0[c - 1], aw.x, aw.y, is_wet(H0[c - 1], b0[c - 1], eps)};
            Nb<T> E{B0[c + 1], b0[c + 1], ae.x, ae.y, is_wet(H0[c + 1], b0[c + 1], eps)};
            Nb<T> S{Bm[c], bm[c], as.x, as.y, is_wet(Hm[c], bm[c], eps)};
            Nb<T> N{Bp[c], bp[c], an.x, an.y, is_wet(Hp[c], bp[c], eps)};
            T ax, ay, phi;
            forces(P, B0[c], b, nm, a0.x, a0.y, W, E, S, N, ax, ay, phi);
            const T den = T(1) + tauT * phi;
            lin_div2(ux, uy, tauT, ax, ay, den, utx, uty);
        }
        T uhx, uhy;
        if constexpr (sizeof(T) == 4) {
            const f2 uh = mul2(mk2(0.5f, 0.5f), add2(mk2(ux, uy), mk2(utx, uty)));
            uhx = uh.x;
            uhy = uh.y;
        } else {
            uhx = T(0.5) * (ux + utx);
            uhy = T(0.5) * (uy + uty);
        }
        T sig = T(0), vx = T(0), vy = T(0);
        while (sp < se && a.src[sp].r < r) ++sp;
        for (int q = sp; q < se && a.src[q].r == r; ++q) {
            if (a.src[q].c == c) {
                sig = (T)(a.src[q].w * s.hq[a.src[q].hydro]);
                vx = (T)a.src[q].vx;
                vy = (T)a.src[q].vy;
            }
        }
        const T ts = tauT * sig;
        T ht, qtx, qty;
        point_source(H, sig, ts, vx, vy, utx, uty, ht, qtx, qty);
        if (P.dist && b < T(WALL_TEST)) distributed_sources(P, tauT, H + ts, utx, uty, ht, qtx, qty);
        const bool wt = is_wet(ht, b, eps);
        T upx, upy;
        div2_if(wt, qtx, qty, ht, upx, upy);
        cA(r)[c] = V4{uhx, uhy, ht, b};
        cB(r)[c] = V4{upx, upy, qtx, qty};
        if (has_src && out_col && r >= HALO && r < HALO + sh) acc_src += (double)ht - (double)H;
    };
    auto ecell = [&](int rr, int col) {
        ECell<T> e;
        const V4 ca = cA(rr)[col];
        const V2 cb2 = reinterpret_cast<const V2*>(&cB(rr)[col])[0];
        e.w[0] = ca.z;
        e.w[1] = ca.x;
        e.w[2] = ca.y;
        e.w[3] = cb2.x;
        e.w[4] = cb2.y;
        e.b = ca.w;
        e.wt = is_wet(e.w[0], e.b, eps);
        return e;
    };
    // S5: MUSCL slopes along x of row r (each cell once; the face fluxes
    // read both sides' slopes)
    auto stage5 = [&](int r) {
        if (!(r >= 5 && r <= nrows - 6 && (cb & 16u))) return;
        T sx[5];
        slopes(ecell(r, c - 1), ecell(r, c), ecell(r, c + 1), sx);
        sX(r)[c] = V4{sx[0], sx[1], sx[3], sx[4]};
    };
    // S4: MUSCL slopes along y and face fluxes of row r (x faces, and the y
    // face below the row)
    auto stage4 = [&](int r) {
        if (!(r >= 4 && r <= nrows - 5 && (cb & 8u))) return;
        const ECell<T> em = ecell(r - 1, c), e0 = ecell(r, c), ep = ecell(r + 1, c);
        T syc[5];
        slopes(em, e0, ep, syc);
        if (r >= 5) face_flux(P, em, syPrev, e0, syc, 2, fyCur[0], fyCur[1], fyCur[2]);
#pragma unroll
        for (int q = 0; q < 5; ++q) syPrev[q] = syc[q];
        if (r >= 5 && r <= nrows - 6 && (cb & 64u)) {
            const ECell<T> x1 = ecell(r, c + 1);
            const V4 xl = sX(r)[c], xr = sX(r)[c + 1];
            const T sL[5] = {xl.x, xl.y, T(0), xl.z, xl.w};
            const T sR[5] = {xr.x, xr.y, T(0), xr.z, xr.w};
            T FH, FQx, FQy;
            face_flux(P, e0, sL, x1, sR, 1, FH, FQx, FQy);
            fX(r)[c] = V4{FQx, FQy, FH, T(0)};
        }
    };
    // S6: final update of row r (K8)
    auto stage6 = [&](int r) {
        if (r >= 5 && r <= nrows - 6 && (cb & 32u)) {
            const V4 fw = fX(r)[c - 1], fe = fX(r)[c];
            T fh = (fw.z - fe.z) + (fyPrev[0] - fyCur[0]);
            T fqx, fqy;
            if constexpr (sizeof(T) == 4) {
                const f2 fq = add2(sub2(mk2(fw.x, fw.y), mk2(fe.x, fe.y)),
                                   sub2(mk2(fyPrev[1], fyPrev[2]), mk2(fyCur[1], fyCur[2])));
                fqx = fq.x;
                fqy = fq.y;
            } else {
                fqx = (fw.x - fe.x) + (fyPrev[1] - fyCur[1]);
                fqy = (fw.y - fe.y) + (fyPrev[2] - fyCur[2]);
            }
            if (a.corr && gx0 + c < a.g.nx + 2 * PAD) {
                // learned sub-grid corrections of the net flux sums, bounded
                // by a fraction of the plain sums when a bound is set
                const size_t gk = (size_t)(gy0 + r) * (size_t)a.g.pitch + (size_t)(gx0 + c);
                const T c0 = a.corr[gk], c1 = a.corr[a.corr_plane + gk], c2 = a.corr[2 * a.corr_plane + gk];
                if (a.corr_bound > T(0)) {
                    const T l0 = a.corr_bound * fabs(fh), l1 = a.corr_bound * fabs(fqx), l2 = a.corr_bound * fabs(fqy);
                    fh = fh + tmin(tmax(c0, -l0), l0);
                    fqx = fqx + tmin(tmax(c1, -l1), l1);
                    fqy = fqy + tmin(tmax(c2, -l2), l2);
                } else {
                    fh += c0;
                    fqx += c1;
                    fqy += c2;
                }
            }
            const V4 ca = cA(r)[c], cb4 = cB(r)[c];
            T hn = ca.z + dth * fh;
            const bool neg = hn < T(0);
            const T hneg = hn;
            hn = neg ? T(0) : hn;
            const bool pos = hn > eps;
            T qxn, qyn;
            if constexpr (sizeof(T) == 4) {
                const f2 qn = fma2(mk2(dth, dth), mk2(fqx, fqy), mk2(cb4.z, cb4.w));
                qxn = pos ? qn.x : T(0);
                qyn = pos ? qn.y : T(0);
            } else {
                qxn = pos ? cb4.z + dth * fqx : T(0);
                qyn = pos ? cb4.w + dth * fqy : T(0);
            }
            const T b = ca.w;
            const bool wetn = is_wet(hn, b, eps);
            T uxn, uyn;
            div2_if(wetn, qxn, qyn, hn, uxn, uyn);
            nS(r)[c] = V4{uxn, uyn, hn, b};
            if (out_col && r >= HALO && r < HALO + sh) {
                const size_t gi = (size_t)(gy0 + r) * (size_t)a.g.pitch + (size_t)(gx0 + c);
                outH[gi] = hn;
                outQx[gi] = qxn;
                outQy[gi] = qyn;
                acc_mass += (double)hn;
                // a clipped negative depth is rare: no FP64 work otherwise
                if (neg) acc_clip += -(double)hneg;
                acc_wet += wetn ? 1 : 0;
                if (a.act) {
                    // stamp the blocks of the new state that hold a wet cell
                    band_wet = band_wet || wetn;
                    const int gy = y0 + r - HALO;
                    if ((gy & ((1 << ACT_LY) - 1)) == (1 << ACT_LY) - 1 || r == HALO + sh - 1) {
                        if (band_wet)
                            a.act[(size_t)(gy >> ACT_LY) * a.act_nbx + ((x0 + c - HALO) >> ACT_LX)] = step + 1;
                        band_wet = false;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) fyPrev[q] = fyCur[q];
    };
    // S7: signal speed of the new state at row r (next step's K3); with ACC
    // also its accelerations for the next step's predictor.  The new state
    // carries b, so no input row older than S3's is needed.
    auto stage7 = [&](int r) {
        if (!(r >= HALO && r < HALO + sh && out_col)) return;
        const V4* N0 = nS(r);
        const V4 n0 = N0[c];
        const T H = n0.z, b = n0.w;
        T ax = T(0), ay = T(0);
        if (is_wet(H, b, eps)) {
            const T ux = n0.x, uy = n0.y;
            const V4 nw = N0[c - 1], ne = N0[c + 1], ns = nS(r - 1)[c], nn = nS(r + 1)[c];
            Nb<T> W{nw.z, nw.w, nw.x, nw.y, is_wet(nw.z, nw.w, eps)};
            Nb<T> E{ne.z, ne.w, ne.x, ne.y, is_wet(ne.z, ne.w, eps)};
            Nb<T> S{ns.z, ns.w, ns.x, ns.y, is_wet(ns.z, ns.w, eps)};
            Nb<T> N{nn.z, nn.w, nn.x, nn.y, is_wet(nn.z, nn.w, eps)};
            accel(P, H, b, ux, uy, W, E, S, N, ax, ay);
            const T v = cell_speed(P, H, ux, uy, ax, ay);
            const bool fin = v <= T(sizeof(T) == 4 ? FLT_MAX : DBL_MAX);
            bad = bad || !fin;
            if constexpr (OPEN) {
                // with an open ring the edge cells' speeds depend on the
                // next fill: the band pass after it supplies them
                const int gy = y0 + r - HALO, gx = x0 + c - HALO;
                const bool edge = gy == 0 || gy == a.g.ny - 1 || gx == 0 || gx == a.g.nx - 1;
                vmax = (fin && !edge && v > vmax) ? v : vmax;
            } else {
                vmax = (fin && v > vmax) ? v : vmax;
            }
        }
        if (ACC) {
            const size_t gi = (size_t)(gy0 + r) * (size_t)a.g.pitch + (size_t)(gx0 + c);
            a.g.A[buf ^ 1][0][gi] = ax;
            a.g.A[buf ^ 1][1][gi] = ay;
        }
    };

    if (skip) {
        if (out_col && !still) {
            if (groupL) {
                for (int r = HALO; r < HALO + sh; ++r) {
                    const size_t gi = (size_t)(gy0 + r) * (size_t)a.g.pitch + (size_t)(gx0 + c);
                    outQx[gi] = T(0);
                    outQy[gi] = T(0);
                    if (ACC) {
                        a.g.A[buf ^ 1][0][gi] = T(0);
                        a.g.A[buf ^ 1][1][gi] = T(0);
                    }
                }
            } else {
                // H^{n+1} = max(0, H + tau*0) + (tau/h)*(+0): H, with -0 turned
                // into +0 (tested on the bits, as fast math may drop the + 0)
                const T* inH = a.g.H[buf];
                for (int r = HALO; r < HALO + sh; ++r) {
                    const size_t gi = (size_t)(gy0 + r) * (size_t)a.g.pitch + (size_t)(gx0 + c);
                    const T H = inH[gi];
                    const T hn = is_neg_zero(H) ? T(0) : H;
                    outH[gi] = hn;
                    acc_mass += (double)hn;
                }
            }
        }
    } else {
    for (int k = 0; k <= nrows + LG::S7 - HALO - 1; ++k) {
        if (k < nrows) {
            if (tid == 0 && k + PREF < nrows) {
                fence_proxy_async();
                issue_row<T, ACC>(s, a, buf, k + PREF, gx0, gy0, cbase);
            }
            // the Lagrangian group's threads observe the copy of row k (the
            // Eulerian group reads no input ring); a wait that gives up is
            // reported after the iteration's barrier (the row's values are
            // then garbage, but every index stays in bounds)
            const unsigned gr = cbase + (unsigned)k;
            if (groupL && !mbar_wait_bounded(&s.bar[gr % NBAR], (gr / NBAR) & 1u)) s.abort = 1;
        }
        if (ACC) {
            if (groupL) {
                stage0(k);
                stage2(k - LG::S2);
                stage3(k - LG::S3);
                stage7(k - LG::S7);
            } else {
                stage5(k - LG::S5);
                stage4(k - LG::S4);
                stage6(k - LG::S6);
            }
        } else {
            if (groupL) {
                stage0(k);
                stage1(k - LG::S1);
                stage2(k - LG::S2);
                stage3(k - LG::S3);
                stage5(k - LG::S5);
            } else {
                stage4(k - LG::S4);
                stage6(k - LG::S6);
                stage7(k - LG::S7);
            }
        }
        __syncthreads();
        if (s.abort) {
            if (tid == 0) atomicOr(&a.ctl->err, (unsigned)ERR_TIMEOUT);
            return false;
        }
    }
    cbase += (unsigned)nrows;
    }

    // per-CTA partials, the next step's signal speed, and the step report
    const double bmax = block_max<NT>((double)vmax, s.red);
    const double bmass = block_sum<NT>(acc_mass, s.red);
    const double bsrc = block_sum<NT>(acc_src, s.red);
    const double bclip = block_sum<NT>(acc_clip, s.red);
    const double bwet = block_sum<NT>((double)acc_wet, s.red);
    const int anybad = __syncthreads_or(bad);
    if (tid == 0) {
        Part p;
        p.mass = bmass;
        p.src = bsrc;
        p.clip = bclip;
        p.wet = (int)bwet;
        p.skipped = skip ? 1 : 0;
        if (!still) a.parts[item] = p;
        if (a.hist) a.hist[item] = (unsigned char)(((hprev << 1) | (skip ? 1u : 0u)) & 3u);
        if (anybad) atomicOr(&a.ctl->err, (unsigned)ERR_NONFINITE);
        atomicMax(&a.ctl->smax[buf ^ 1], (unsigned long long)__double_as_longlong(bmax));
        __threadfence();
        const unsigned ticket = atomicAdd(&a.ctl->done, 1u);
        s.last = (ticket == (unsigned)a.nitems - 1u);
    }
    __syncthreads();
    if (s.last) {
        __threadfence();
        double m = 0.0, sr = 0.0, cl = 0.0, w = 0.0, sk = 0.0;
        for (int i = tid; i < a.nitems; i += NT) {
            m += __ldcg(&a.parts[i].mass);
            sr += __ldcg(&a.parts[i].src);
            cl += __ldcg(&a.parts[i].clip);
            w += (double)__ldcg(&a.parts[i].wet);
            sk += (double)__ldcg(&a.parts[i].skipped);
        }
        m = block_sum<NT>(m, s.red);
        sr = block_sum<NT>(sr, s.red);
        cl = block_sum<NT>(cl, s.red);
        w = block_sum<NT>(w, s.red);
        sk = block_sum<NT>(sk, s.red);
        if (tid == 0) {
            const double h = (double)P.h;
            Ctl* ctl = a.ctl;
            ctl->mass = m * h * h;
            ctl->src_vol = sr * h * h;
            ctl->clip_vol = cl * h * h;
            ctl->wet = (long long)w;
            ctl->skipped = (long long)sk;
            ctl->tau_last = (double)tauT;
            ctl->t = step_time_after(ctl, a.sp, buf, (double)tauT);
            ctl->max_speed = __longlong_as_double((long long)atomicAdd(&ctl->smax[buf ^ 1], 0ull));
            ctl->smax[buf] = 0ull;
            ctl->step = step + 1;
            ctl->done = 0u;
            __threadfence();
        }
    }
    __syncthreads();
    return true;
}

template <class T, bool ACC>
__device__ __forceinline__ FSmem<T, ACC>& fused_smem() {
    // Round up to 128 bytes (TMA destinations) by offsetting into the shared
    // array itself: the compiler then still knows every access is to shared
    // memory (32-bit LDS/STS addressing instead of generic 64-bit loads).
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const unsigned off = (128u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u;
    return *reinterpret_cast<FSmem<T, ACC>*>(smem_raw + off);
}

template <class T, bool ACC>
__device__ __forceinline__ void fused_init_barriers(FSmem<T, ACC>& s) {
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NBAR; ++i) mbar_init(&s.bar[i], 1);
        s.abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
}

// One grid: CTA b runs work item b.  OPEN: the grid has an open
// (zero-gradient) ghost ring, whose band pass supplies the edge cells'
// signal speeds.
template <class T, bool ACC, bool OPEN = false>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1) k_fused(const __grid_constant__ FusedArgs<T> a) {
    FSmem<T, ACC>& s = fused_smem<T, ACC>();
    fused_init_barriers(s);
    unsigned cbase = 0;
    fused_item<T, ACC, OPEN>(s, a, blockIdx.x, cbase);
}

// Many grids in one persistent launch (batched ensemble): CTAs take
// (scenario, item) entries from a device work list until it is exhausted;
// each scenario keeps its own time, time step, sources, walls and report.
// Every scenario is a context, so accelerations are stored (ACC).
template <class T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1) k_fused_batch(const __grid_constant__ BatchArgs<T> b) {
    FSmem<T, true>& s = fused_smem<T, true>();
    fused_init_barriers(s);
    unsigned cbase = 0;
    while (true) {
        if (threadIdx.x == 0) s.witem = (int)atomicAdd(&b.bc->next, 1u);
        __syncthreads();
        const int w = s.witem;
        __syncthreads();
        if (w >= b.nwork) break;
        const int2 e = b.work[w];
        if (!fused_item<T, true>(s, b.descs[e.x], e.y, cbase)) break;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&b.bc->exited, 1u) == gridDim.x - 1u) {
            b.bc->next = 0u;
            b.bc->exited = 0u;
            __threadfence();
        }
    }
}

// Opt the fused kernel into its shared-memory size; returns CTAs per SM.
template <class T>
cudaError_t prepare_fused(int* ctas_per_sm) {
    const size_t smem = fused_smem_bytes_v<T, true>();
    cudaError_t e = cudaFuncSetAttribute(k_fused<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fused_smem_bytes_v<T, false>());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_fused<T, true>, NT, smem);
}

template <class T>
cudaError_t prepare_fused_batch(int* ctas_per_sm) {
    const size_t smem = fused_smem_bytes<T>();
    cudaError_t e = cudaFuncSetAttribute(k_fused_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_fused_batch<T>, NT, smem);
}

template <class T>
cudaError_t launch_fused_batch(const BatchArgs<T>& b, int grid, cudaStream_t st) {
    k_fused_batch<T><<<grid, NT, fused_smem_bytes<T>(), st>>>(b);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_fused(const FusedArgs<T>& a, cudaStream_t st) {
    if (a.g.A[0][0] && a.open_ring) k_fused<T, true, true><<<a.nitems, NT, fused_smem_bytes_v<T, true>(), st>>>(a);
    else if (a.g.A[0][0]) k_fused<T, true><<<a.nitems, NT, fused_smem_bytes_v<T, true>(), st>>>(a);
    else k_fused<T, false><<<a.nitems, NT, fused_smem_bytes_v<T, false>(), st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ staged kernels

template <class T>
struct PAcc {
    int pitch;
    __device__ __forceinline__ size_t operator()(int i, int j) const {
        return (size_t)(j + PAD) * (size_t)pitch + (size_t)(i + PAD);
    }
};

__device__ __forceinline__ int ctl_buf(const Ctl* ctl) {
    return (int)(*(volatile const long long*)&ctl->step & 1);
}

// Rows per block of the kernels that reduce FP64 budgets (speed pass,
// corrector, final update): 32 columns x SPEED_ROWS rows, 8 rows per thread.
constexpr int SPEED_ROWS = 64;

// tau_n for a staged kernel, evaluated once per block: it is an FP64
// division, and a warp-wide FP64 instruction holds this part's FP64 pipe for
// 16 cycles, so evaluating it per cell cost each stage ~0.4 ms per 4096^2
// launch.  Every thread of the block must call it (it synchronises).
template <class T>
__device__ __forceinline__ T block_tau(const StagedArgs<T>& a) {
    __shared__ double st;
    if (threadIdx.x == 0 && threadIdx.y == 0) st = step_tau(a.ctl, a.sp, ctl_buf(a.ctl));
    __syncthreads();
    return (T)st;
}

template <class T>
__device__ __forceinline__ Nb<T> nb_at(const StagedArgs<T>& a, const T* Hwet, const T* hs, const T* ux,
                                       const T* uy, size_t k) {
    Nb<T> n;
    n.hs = hs[k];
    n.b = a.g.b[k];
    n.ux = ux[k];
    n.uy = uy[k];
    n.wet = is_wet(Hwet[k], n.b, a.P.eps);
    return n;
}

template <class T>
__global__ void ks_prim(const StagedArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.g.nx || j >= a.g.ny) return;
    const int buf = ctl_buf(a.ctl);
    const size_t k = PAcc<T>{a.g.pitch}(i, j);
    const T H = a.g.H[buf][k];
    const bool wet = is_wet(H, a.g.b[k], a.P.eps);
    a.ux[k] = wet ? a.g.Qx[buf][k] / H : T(0);
    a.uy[k] = wet ? a.g.Qy[buf][k] / H : T(0);
}

// forces from depth hs and velocity (ux, uy); wet mask of the state at t_n
template <class T>
__global__ void ks_forces(const StagedArgs<T> a, int second) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.g.nx || j >= a.g.ny) return;
    const int buf = ctl_buf(a.ctl);
    const PAcc<T> at{a.g.pitch};
    const size_t k = at(i, j);
    const T* Hw = a.g.H[buf];
    const T* hs = second ? a.hs : Hw;
    const T* ux = second ? a.usx : a.ux;
    const T* uy = second ? a.usy : a.uy;
    T* ax = second ? a.ax2 : a.ax;
    T* ay = second ? a.ay2 : a.ay;
    T* phi = second ? a.phi2 : a.phi;
    if (!is_wet(Hw[k], a.g.b[k], a.P.eps)) {
        ax[k] = T(0); ay[k] = T(0); phi[k] = T(0);
        return;
    }
    const Nb<T> W = nb_at(a, Hw, hs, ux, uy, at(i - 1, j)), E = nb_at(a, Hw, hs, ux, uy, at(i + 1, j));
    const Nb<T> S = nb_at(a, Hw, hs, ux, uy, at(i, j - 1)), N = nb_at(a, Hw, hs, ux, uy, at(i, j + 1));
    T fx, fy, fp;
    forces(a.P, hs[k], a.g.b[k], a.g.n[k], ux[k], uy[k], W, E, S, N, fx, fy, fp);
    ax[k] = fx; ay[k] = fy; phi[k] = fp;
}

template <class T>
__global__ void ks_predict(const StagedArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const T tauT = block_tau(a);
    if (i >= a.g.nx || j >= a.g.ny) return;
    const int buf = ctl_buf(a.ctl);
    const T th = T(0.5) * tauT;
    const size_t k = PAcc<T>{a.g.pitch}(i, j);
    T usx = T(0), usy = T(0);
    if (is_wet(a.g.H[buf][k], a.g.b[k], a.P.eps)) {
        const T den = T(1) + th * a.phi[k];
        usx = (a.ux[k] + th * a.ax[k]) / den;
        usy = (a.uy[k] + th * a.ay[k]) / den;
    }
    a.usx[k] = usx;
    a.usy[k] = usy;
}

template <class T>
__global__ void ks_hstar(const StagedArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const T tauT = block_tau(a);
    if (i >= a.g.nx || j >= a.g.ny) return;
    const int buf = ctl_buf(a.ctl);
    const T th = T(0.5) * tauT;
    const PAcc<T> at{a.g.pitch};
    const size_t k = at(i, j);
    const T H = a.g.H[buf][k];
    T hs = H;
    if (is_wet(H, a.g.b[k], a.P.eps)) {
        const T u = a.usx[k], uW = a.usx[at(i - 1, j)], uE = a.usx[at(i + 1, j)];
        const T v = a.usy[k], vS = a.usy[at(i, j - 1)], vN = a.usy[at(i, j + 1)];
        const T fxm = T(0.5) * (uW + u), fxp = T(0.5) * (u + uE);
        const T fym = T(0.5) * (vS + v), fyp = T(0.5) * (v + vN);
        const T D = ((fxp - fxm) + (fyp - fym)) / a.P.h;
        hs = H / tmax(T(0.5), T(1) + th * D);
    }
    a.hs[k] = hs;
}

template <class T>
__global__ void ks_sources(const StagedArgs<T> a) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.nsrc) return;
    const int buf = ctl_buf(a.ctl);
    const T tauT = (T)step_tau(a.ctl, a.sp, buf);
    const double q = hydro_value(a.hydro + 4 * a.s_hydro[m], a.ctl->t + 0.5 * (double)tauT);
    const int k = a.s_cell[m];
    a.sig[k] = (T)(a.s_w[m] * q);
    a.svx[k] = (T)a.s_vx[m];
    a.svy[k] = (T)a.s_vy[m];
}

template <class T>
__global__ void ks_correct(const StagedArgs<T> a) {
    // a block covers 32 columns x SPEED_ROWS rows (each thread SPEED_ROWS / 8
    // rows), so the FP64 source budget is reduced once per 2048 cells
    __shared__ double red[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int jend = min(a.g.ny, (int)(blockIdx.y + 1) * SPEED_ROWS);
    double src = 0.0;
    const T tauT = block_tau(a);
    if (i < a.g.nx)
    for (int j = blockIdx.y * SPEED_ROWS + threadIdx.y; j < jend; j += 8) {
        const int buf = ctl_buf(a.ctl);
        const size_t k = PAcc<T>{a.g.pitch}(i, j);
        const T H = a.g.H[buf][k], b = a.g.b[k];
        T utx = T(0), uty = T(0);
        if (is_wet(H, b, a.P.eps)) {
            const T den = T(1) + tauT * a.phi2[k];
            utx = (a.ux[k] + tauT * a.ax2[k]) / den;
            uty = (a.uy[k] + tauT * a.ay2[k]) / den;
        }
        a.utx[k] = utx;
        a.uty[k] = uty;
        a.uhx[k] = T(0.5) * (a.ux[k] + utx);
        a.uhy[k] = T(0.5) * (a.uy[k] + uty);
        const T sig = a.sig[k];
        const T ts = tauT * sig;
        T ht, qtx, qty;
        point_source(H, sig, ts, a.svx[k], a.svy[k], utx, uty, ht, qtx, qty);
        if (a.P.dist && b < T(WALL_TEST)) distributed_sources(a.P, tauT, H + ts, utx, uty, ht, qtx, qty);
        const bool wt = is_wet(ht, b, a.P.eps);
        a.ht[k] = ht;
        a.qtx[k] = qtx;
        a.qty[k] = qty;
        a.upx[k] = wt ? qtx / ht : T(0);
        a.upy[k] = wt ? qty / ht : T(0);
        src += (double)ht - (double)H;
    }
    const double s = block_sum<256>(src, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) a.parts2[blockIdx.y * gridDim.x + blockIdx.x].src = s;
}

template <class T>
__device__ __forceinline__ ECell<T> ecell_at(const StagedArgs<T>& a, size_t k) {
    ECell<T> e;
    const T ht = a.ht[k], bb = a.g.b[k];
    e.w[0] = ht;
    e.w[1] = a.uhx[k];
    e.w[2] = a.uhy[k];
    e.w[3] = a.upx[k];
    e.w[4] = a.upy[k];
    e.b = bb;
    e.wt = is_wet(ht, bb, a.P.eps);
    return e;
}

// fluxes of the faces i+1/2 (dir 0, i in [-1, nx-1]) or j+1/2 (dir 1)
template <class T>
__global__ void ks_flux(const StagedArgs<T> a, int dir) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x - (dir == 0 ? 1 : 0);
    const int j = blockIdx.y * blockDim.y + threadIdx.y - (dir == 1 ? 1 : 0);
    if (i >= a.g.nx || j >= a.g.ny) return;
    const PAcc<T> at{a.g.pitch};
    const int di = dir == 0 ? 1 : 0, dj = dir == 1 ? 1 : 0;
    const ECell<T> l2 = ecell_at(a, at(i - di, j - dj)), l = ecell_at(a, at(i, j));
    const ECell<T> r = ecell_at(a, at(i + di, j + dj)), r2 = ecell_at(a, at(i + 2 * di, j + 2 * dj));
    T sL[5], sR[5];
    slopes(l2, l, r, sL);
    slopes(l, r, r2, sR);
    T FH, FQx, FQy;
    face_flux(a.P, l, sL, r, sR, dir == 0 ? 1 : 2, FH, FQx, FQy);
    T* const* f = dir == 0 ? a.fx : a.fy;
    const size_t k = at(i, j);
    f[0][k] = FH;
    f[1][k] = FQx;
    f[2][k] = FQy;
}

template <class T>
__global__ void ks_final(const StagedArgs<T> a) {
    // 32 columns x SPEED_ROWS rows per block, as ks_correct
    __shared__ double red[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int jend = min(a.g.ny, (int)(blockIdx.y + 1) * SPEED_ROWS);
    double mass = 0.0, clip = 0.0;
    int wet = 0;
    const T tauT = block_tau(a);
    if (i < a.g.nx)
    for (int j = blockIdx.y * SPEED_ROWS + threadIdx.y; j < jend; j += 8) {
        const int buf = ctl_buf(a.ctl);
        const T dth = tauT / a.P.h;
        const PAcc<T> at{a.g.pitch};
        const size_t k = at(i, j), kw = at(i - 1, j), ks = at(i, j - 1);
        const T fh = (a.fx[0][kw] - a.fx[0][k]) + (a.fy[0][ks] - a.fy[0][k]);
        const T fqx = (a.fx[1][kw] - a.fx[1][k]) + (a.fy[1][ks] - a.fy[1][k]);
        const T fqy = (a.fx[2][kw] - a.fx[2][k]) + (a.fy[2][ks] - a.fy[2][k]);
        T hn = a.ht[k] + dth * fh;
        if (hn < T(0)) {
            clip += -(double)hn;
            hn = T(0);
        }
        T qxn = T(0), qyn = T(0);
        if (hn > a.P.eps) {
            qxn = a.qtx[k] + dth * fqx;
            qyn = a.qty[k] + dth * fqy;
        }
        a.g.H[buf ^ 1][k] = hn;
        a.g.Qx[buf ^ 1][k] = qxn;
        a.g.Qy[buf ^ 1][k] = qyn;
        mass += (double)hn;
        wet += is_wet(hn, a.g.b[k], a.P.eps) ? 1 : 0;
    }
    const int bl = blockIdx.y * gridDim.x + blockIdx.x;
    const double m = block_sum<256>(mass, red);
    const double c = block_sum<256>(clip, red);
    const double w = block_sum<256>((double)wet, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        a.parts[bl].mass = m;
        a.parts[bl].clip = c;
        a.parts[bl].wet = (int)w;
    }
}

// Signal speed (and mass) of the state in buffer `which` (0: current,
// 1: next); atomicMax into the smax slot of that state's step parity.
// Where the grid stores accelerations, also writes them for that state.
// [i0, i1) x [j0, j1): the cells the launch covers (a region of the grid);
// parts = 0 leaves the per-block partial sums alone.
// A block of 32 x 8 threads covers 32 columns x SPEED_ROWS rows (each
// thread SPEED_ROWS / 8 rows): the speed max is kept in T (a max is exact
// in any precision) and the wet count as an integer, so FP64 work (slow on
// this part) is one conversion and one add per cell for the mass plus one
// set of block reductions per SPEED_ROWS * 32 cells.

template <class T>
__global__ void ks_speed(const StagedArgs<T> a, int which, int i0 = 0, int j0 = 0, int parts = 1,
                         int i1 = INT_MAX, int j1 = INT_MAX, int check = 0) {
    __shared__ double red[8];
    const int i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    const int jb = j0 + blockIdx.y * SPEED_ROWS + threadIdx.y;
    const int jend = min(min(a.g.ny, j1), j0 + (int)(blockIdx.y + 1) * SPEED_ROWS);
    const int buf = ctl_buf(a.ctl) ^ which;
    const long long stamp = *(volatile const long long*)&a.ctl->step + which;
    T vmax = T(0);
    double mass = 0.0;
    int wet = 0;
    bool bad = false, neg = false;
    const PAcc<T> at{a.g.pitch};
    const T* Hs = a.g.H[buf];
    const T* Qx = a.g.Qx[buf];
    const T* Qy = a.g.Qy[buf];
    const T eps = a.P.eps;
    auto nb = [&](size_t k) {
        Nb<T> n;
        n.hs = Hs[k];
        n.b = a.g.b[k];
        n.wet = is_wet(n.hs, n.b, eps);
        // the fused kernel's form of U = Q/H, so a state set from the host
        // gets the stored forces the kernel would have stored
        div2_if(n.wet, Qx[k], Qy[k], n.hs, n.ux, n.uy);
        return n;
    };
    if (i < a.g.nx && i < i1) {
        for (int j = jb; j < jend; j += 8) {
            const size_t k = at(i, j);
            const Nb<T> C = nb(k);
            mass += (double)C.hs;
            if (check) {
                // a state just copied in: non-finite H, Qx or Qy (bit 0);
                // negative depth (bit 1; not NaN, not -0)
                bad = bad || nonfinite_bits(C.hs) || nonfinite_bits(Qx[k]) || nonfinite_bits(Qy[k]);
                neg = neg || C.hs < T(0);
            } else if (!(C.hs >= T(0) && C.hs <= T(sizeof(T) == 4 ? FLT_MAX : DBL_MAX))) {
                bad = true;
            }
            T ax = T(0), ay = T(0);
            if (C.wet) {
                ++wet;
                if (a.act) a.act[(size_t)(j >> ACT_LY) * a.act_nbx + (i >> ACT_LX)] = stamp;
                accel(a.P, C.hs, C.b, C.ux, C.uy, nb(at(i - 1, j)), nb(at(i + 1, j)), nb(at(i, j - 1)),
                      nb(at(i, j + 1)), ax, ay);
                const T v = cell_speed(a.P, C.hs, C.ux, C.uy, ax, ay);
                const bool fin = v <= T(sizeof(T) == 4 ? FLT_MAX : DBL_MAX);
                bad = bad || !fin;
                // open ring: the edge cells' speeds come from the band pass
                const bool edge = a.open_ring && (i == 0 || i == a.g.nx - 1 || j == 0 || j == a.g.ny - 1);
                vmax = (fin && !edge && v > vmax) ? v : vmax;
            }
            if (a.g.A[buf][0]) {
                a.g.A[buf][0][k] = ax;
                a.g.A[buf][1][k] = ay;
            }
        }
    }
    const double bm = block_max<256>((double)vmax, red);
    const double bs = block_sum<256>(mass, red);
    const double bw = block_sum<256>((double)wet, red);
    const int anybad = __syncthreads_or(bad);
    const int anyneg = __syncthreads_or(neg);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int bl = blockIdx.y * gridDim.x + blockIdx.x;
        const int slot = (int)(stamp & 1);
        atomicMax(&a.ctl->smax[slot], (unsigned long long)__double_as_longlong(bm));
        if (anybad) atomicOr(&a.ctl->err, (unsigned)ERR_NONFINITE);
        if (anyneg) atomicOr(&a.ctl->err, 2u);
        if (which == 0 && parts) {
            a.parts[bl].mass = bs;
            a.parts[bl].wet = (int)bw;
        }
    }
}

// Stored accelerations (a_x, a_y) of the current state on the band a
// ghost-ring fill changes: ring cells within HALO of the interior (the
// fused kernel's predictor reads them) and the first interior row and
// column (their forces see the ring).  Four strips of width HALO + 1 over
// a linear index; no speed or mass report (the ring is not part of either).
template <class T>
__global__ void k_band_acc(const StagedArgs<T> a) {
    constexpr int B = HALO + 1;
    const int W = a.g.nx + 2 * HALO;
    const long long ntop = (long long)B * W;
    const long long nside = (long long)max(0, a.g.ny - 2) * B;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i, j;
    if (idx < ntop) {
        j = -HALO + (int)(idx / W);
        i = -HALO + (int)(idx % W);
    } else if ((idx -= ntop) < ntop) {
        j = a.g.ny - 1 + (int)(idx / W);
        i = -HALO + (int)(idx % W);
    } else if ((idx -= ntop) < nside) {
        j = 1 + (int)(idx / B);
        i = -HALO + (int)(idx % B);
    } else if ((idx -= nside) < nside) {
        j = 1 + (int)(idx / B);
        i = a.g.nx - 1 + (int)(idx % B);
    } else {
        return;
    }
    const int buf = ctl_buf(a.ctl);
    const PAcc<T> at{a.g.pitch};
    const T* Hs = a.g.H[buf];
    const T* Qx = a.g.Qx[buf];
    const T* Qy = a.g.Qy[buf];
    const T eps = a.P.eps;
    auto nb = [&](size_t k) {
        Nb<T> n;
        n.hs = Hs[k];
        n.b = a.g.b[k];
        n.wet = is_wet(n.hs, n.b, eps);
        // the fused kernel's form of U = Q/H, so a state set from the host
        // gets the stored forces the kernel would have stored
        div2_if(n.wet, Qx[k], Qy[k], n.hs, n.ux, n.uy);
        return n;
    };
    const size_t k = at(i, j);
    const Nb<T> C = nb(k);
    T ax = T(0), ay = T(0);
    if (C.wet)
        accel(a.P, C.hs, C.b, C.ux, C.uy, nb(at(i - 1, j)), nb(at(i + 1, j)), nb(at(i, j - 1)), nb(at(i, j + 1)),
              ax, ay);
    a.g.A[buf][0][k] = ax;
    a.g.A[buf][1][k] = ay;
    if (a.open_ring && C.wet) {
        // the step's signal speed over the state the fill completed: the
        // edge cells and the ring (along a normal every ring cell repeats
        // the state and forces of the one at distance 1, so distances up to
        // HALO cover the whole ring)
        const T v = cell_speed(a.P, C.hs, C.ux, C.uy, ax, ay);
        if (!(v <= T(sizeof(T) == 4 ? FLT_MAX : DBL_MAX))) atomicOr(&a.ctl->err, (unsigned)ERR_NONFINITE);
        else atomicMax(&a.ctl->smax[buf], (unsigned long long)__double_as_longlong((double)v));
    }
}

template <class T>
cudaError_t launch_band_acc(const StagedArgs<T>& a, cudaStream_t st) {
    const long long n = 2LL * (HALO + 1) * (a.g.nx + 2 * HALO) + 2LL * std::max(0, a.g.ny - 2) * (HALO + 1);
    k_band_acc<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T>
dim3 speed_grid(int ni, int nj) {
    return dim3((ni + 31) / 32, (nj + SPEED_ROWS - 1) / SPEED_ROWS);
}

// Reduce the partials of a staged step (fixed order) and advance the control
// block; with init != 0 only report the mass of the current state.
template <class T>
__global__ void ks_finish(const StagedArgs<T> a, int nblocks, int init) {
    // a state set from the host: no work item has a skip history
    if (init && a.hist)
        for (int i = threadIdx.x; i < a.nhist; i += 256) a.hist[i] = 0;
    __shared__ double red[8];
    double m = 0.0, sr = 0.0, cl = 0.0, w = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 256) {
        m += a.parts[i].mass;
        w += (double)a.parts[i].wet;
        if (!init) {
            sr += a.parts2[i].src;
            cl += a.parts[i].clip;
        }
    }
    m = block_sum<256>(m, red);
    sr = block_sum<256>(sr, red);
    cl = block_sum<256>(cl, red);
    w = block_sum<256>(w, red);
    if (threadIdx.x == 0) {
        Ctl* ctl = a.ctl;
        const double h = (double)a.P.h;
        ctl->mass = m * h * h;
        ctl->wet = (long long)w;
        ctl->skipped = 0;
        if (!init) {
            const int buf = (int)(ctl->step & 1);
            const T tauT = (T)step_tau(ctl, a.sp, buf);
            ctl->src_vol = sr * h * h;
            ctl->clip_vol = cl * h * h;
            ctl->tau_last = (double)tauT;
            ctl->t = step_time_after(ctl, a.sp, buf, (double)tauT);
            ctl->max_speed = __longlong_as_double((long long)ctl->smax[buf ^ 1]);
            ctl->smax[buf] = 0ull;
            ctl->step = ctl->step + 1;
        } else {
            ctl->max_speed = __longlong_as_double((long long)ctl->smax[ctl->step & 1]);
        }
    }
}

template <class T>
cudaError_t launch_staged(const StagedArgs<T>& a, cudaStream_t st) {
    const dim3 blk(32, 8);
    const dim3 grd((a.g.nx + 31) / 32, (a.g.ny + 7) / 8);
    const dim3 grdx((a.g.nx + 1 + 31) / 32, (a.g.ny + 7) / 8);
    const dim3 grdy((a.g.nx + 31) / 32, (a.g.ny + 1 + 7) / 8);
    // the budget kernels (corrector, final update) run 32 x SPEED_ROWS blocks
    const dim3 grdb = speed_grid<T>(a.g.nx, a.g.ny);
    const int nblocks = (int)(grdb.x * grdb.y);
    const size_t plane = (size_t)a.g.pitch * (size_t)(a.g.ny + 2 * PAD) * sizeof(T);
    ks_prim<T><<<grd, blk, 0, st>>>(a);
    ks_forces<T><<<grd, blk, 0, st>>>(a, 0);
    ks_predict<T><<<grd, blk, 0, st>>>(a);
    ks_hstar<T><<<grd, blk, 0, st>>>(a);
    ks_forces<T><<<grd, blk, 0, st>>>(a, 1);
    cudaMemsetAsync(a.sig, 0, plane, st);
    cudaMemsetAsync(a.svx, 0, plane, st);
    cudaMemsetAsync(a.svy, 0, plane, st);
    if (a.nsrc > 0) ks_sources<T><<<(a.nsrc + 127) / 128, 128, 0, st>>>(a);
    ks_correct<T><<<grdb, blk, 0, st>>>(a);
    ks_flux<T><<<grdx, blk, 0, st>>>(a, 0);
    ks_flux<T><<<grdy, blk, 0, st>>>(a, 1);
    ks_final<T><<<grdb, blk, 0, st>>>(a);
    ks_speed<T><<<speed_grid<T>(a.g.nx, a.g.ny), blk, 0, st>>>(a, 1);
    ks_finish<T><<<1, 256, 0, st>>>(a, nblocks, 0);
    return cudaGetLastError();
}

static __global__ void k_zero_cur_slot(Ctl* ctl) { ctl->smax[ctl->step & 1] = 0ull; }

// Signal speed and stored accelerations of the current state over the cells
// [i0, i0 + ni) x [j0, j0 + nj) only (after a change confined to them): the
// step's speed slot takes the max with it, which can only over-estimate.
template <class T>
cudaError_t launch_state_speed_region(const StagedArgs<T>& a, int i0, int j0, int ni, int nj, cudaStream_t st) {
    const dim3 blk(32, 8);
    ks_speed<T><<<speed_grid<T>(ni, nj), blk, 0, st>>>(a, 0, i0, j0, 0, i0 + ni, j0 + nj);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_state_speed(const StagedArgs<T>& a, cudaStream_t st, int check) {
    const dim3 blk(32, 8);
    const dim3 grd = speed_grid<T>(a.g.nx, a.g.ny);
    k_zero_cur_slot<<<1, 1, 0, st>>>(a.ctl);
    ks_speed<T><<<grd, blk, 0, st>>>(a, 0, 0, 0, 1, INT_MAX, INT_MAX, check);
    ks_finish<T><<<1, 256, 0, st>>>(a, (int)(grd.x * grd.y), 1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host copies

// FP64 host layout -> padded field.  With flag != nullptr, values that are
// not finite (bit 0) or negative (bit 1, when check_neg) are reported there.
template <class T>
__global__ void k_pack(const double* __restrict__ src, T* __restrict__ dst, int nx, int ny, int pitch,
                       unsigned* flag, int check_neg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i < nx) {
        const double v = src[(size_t)j * nx + i];
        const T tv = (T)v;
        dst[(size_t)(j + PAD) * pitch + (i + PAD)] = tv;
        if (flag) {
            // the checks on the bits (integer work; FP64 compares are slow on
            // this part): v infinite or NaN, or its rounding to T overflows
            // (bit 0); v < 0, i.e. negative, not NaN and not -0 (bit 1)
            const unsigned long long vb = (unsigned long long)__double_as_longlong(v);
            const bool vnf = (vb & 0x7FF0000000000000ull) == 0x7FF0000000000000ull;
            const bool vnan = vnf && (vb & 0x000FFFFFFFFFFFFFull) != 0ull;
            unsigned bad = (vnf || nonfinite_bits(tv)) ? 1u : 0u;
            if (check_neg && (vb >> 63) && !vnan && (vb << 1) != 0ull) bad |= 2u;
            if (__any_sync(__activemask(), bad != 0) && bad) atomicOr(flag, bad);
        }
    }
}

// FP64 host layout of the whole padded extent (ring included) -> padded
// field.
template <class T>
__global__ void k_pack_full(const double* __restrict__ src, T* __restrict__ dst, int nxe, int pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i < nxe) dst[(size_t)j * pitch + i] = (T)src[(size_t)j * nxe + i];
}

__device__ __forceinline__ int floor_div4(int i) { return i >= 0 ? i / 4 : -((3 - i) / 4); }

// Two-level grid system (Sec. 2.2, Fig. 1): the ghost ring of a fine patch
// (4x finer, its interior cell (0, 0) in coarse cell (ix0, iy0)) from the
// coarse grid, at the fraction w of the coarse step just taken (0: its
// start, the other coarse buffer; 1: its end, the current one).  Each ring
// cell takes the coarse cell containing its centre: the coarse state is
// interpolated linearly in time, the fine depth is the coarse free surface
// above the fine bed (so still water stays still) and the velocity is the
// coarse one.  Dry coarse cells and walls give dry ghosts.
template <class T>
__global__ void k_nest_ring(const Grid<T> f, const Ctl* __restrict__ fctl, const Grid<T> c, const Ctl* __restrict__ cctl,
                            int ix0, int iy0, double w, double eps) {
    // ring cells only: PAD full rows above and below, PAD columns left and
    // right of the interior rows
    const int nxe = f.nx + 2 * PAD;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nband = (long long)PAD * nxe, nside = (long long)f.ny * PAD;
    if (e >= 2 * nband + 2 * nside) return;
    int ip, jp;
    if (e < 2 * nband) {
        const int r = (int)(e / nxe);
        ip = (int)(e % nxe);
        jp = r < PAD ? r : f.ny + r;  // rows 0..PAD-1 and ny+PAD..ny+2PAD-1
    } else {
        const long long q = e - 2 * nband;
        const int r = (int)(q / (2 * PAD)), k = (int)(q % (2 * PAD));
        jp = PAD + r;
        ip = k < PAD ? k : f.nx + k;  // columns 0..PAD-1 and nx+PAD..nx+2PAD-1
    }
    const int i = ip - PAD, j = jp - PAD;
    const int xc = ix0 + floor_div4(i), yc = iy0 + floor_div4(j);
    const int cnew = (int)(*(volatile const long long*)&cctl->step & 1), cold = cnew ^ 1;
    const int fb = (int)(*(volatile const long long*)&fctl->step & 1);
    const size_t kc = (size_t)(yc + PAD) * c.pitch + (size_t)(xc + PAD);
    const size_t kf = (size_t)jp * f.pitch + (size_t)ip;
    const double Hc = (1.0 - w) * (double)c.H[cold][kc] + w * (double)c.H[cnew][kc];
    const double Qxc = (1.0 - w) * (double)c.Qx[cold][kc] + w * (double)c.Qx[cnew][kc];
    const double Qyc = (1.0 - w) * (double)c.Qy[cold][kc] + w * (double)c.Qy[cnew][kc];
    const double bc = (double)c.b[kc], bf = (double)f.b[kf];
    double hg = 0.0, qx = 0.0, qy = 0.0;
    if (Hc > eps && bc < WALL_TEST && bf < WALL_TEST) {
        const double eta = Hc + bc;
        hg = eta - bf > 0.0 ? eta - bf : 0.0;
        qx = hg * (Qxc / Hc);
        qy = hg * (Qyc / Hc);
    }
    f.H[fb][kf] = (T)hg;
    f.Qx[fb][kf] = (T)qx;
    f.Qy[fb][kf] = (T)qy;
}

// Open (outflow) boundary: before a step every ring cell that is not a wall
// (bed below 1e29) takes the state of the nearest interior cell (zero
// gradient across the boundary), so waves and flow leave the domain.
template <class T>
__global__ void k_ring_outflow(const Grid<T> g, const Ctl* __restrict__ ctl) {
    const int nxe = g.nx + 2 * PAD;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nband = (long long)PAD * nxe, nside = (long long)g.ny * PAD;
    if (e >= 2 * nband + 2 * nside) return;
    int ip, jp;
    if (e < 2 * nband) {
        const int r = (int)(e / nxe);
        ip = (int)(e % nxe);
        jp = r < PAD ? r : g.ny + r;
    } else {
        const long long q = e - 2 * nband;
        const int r = (int)(q / (2 * PAD)), k = (int)(q % (2 * PAD));
        jp = PAD + r;
        ip = k < PAD ? k : g.nx + k;
    }
    const size_t kg = (size_t)jp * g.pitch + (size_t)ip;
    if (!(g.b[kg] < T(WALL_TEST))) return;
    const int i = min(max(ip - PAD, 0), g.nx - 1), j = min(max(jp - PAD, 0), g.ny - 1);
    const size_t ki = (size_t)(j + PAD) * g.pitch + (size_t)(i + PAD);
    const int buf = (int)(*(volatile const long long*)&ctl->step & 1);
    g.H[buf][kg] = g.H[buf][ki];
    g.Qx[buf][kg] = g.Qx[buf][ki];
    g.Qy[buf][kg] = g.Qy[buf][ki];
}

// Feedback of a fine patch: each coarse cell it covers takes the means of
// its 4 x 4 fine cells' H, Qx, Qy (summed row by row in the state
// precision), which keeps the patch's water volume and momentum.
template <class T>
__global__ void k_nest_restrict(const Grid<T> f, const Ctl* __restrict__ fctl, const Grid<T> c,
                                const Ctl* __restrict__ cctl, int ix0, int iy0) {
    const int ncx = f.nx / 4, ncy = f.ny / 4;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncx * ncy) return;
    const int u = e % ncx, v = e / ncx;
    const int fb = (int)(*(volatile const long long*)&fctl->step & 1);
    const int cb = (int)(*(volatile const long long*)&cctl->step & 1);
    T sh = T(0), sx = T(0), sy = T(0);
    for (int dy = 0; dy < 4; ++dy)
        for (int dx = 0; dx < 4; ++dx) {
            const size_t k = (size_t)(4 * v + dy + PAD) * f.pitch + (size_t)(4 * u + dx + PAD);
            sh += f.H[fb][k];
            sx += f.Qx[fb][k];
            sy += f.Qy[fb][k];
        }
    const size_t kc = (size_t)(iy0 + v + PAD) * c.pitch + (size_t)(ix0 + u + PAD);
    c.H[cb][kc] = sh * T(0.0625);
    c.Qx[cb][kc] = sx * T(0.0625);
    c.Qy[cb][kc] = sy * T(0.0625);
}

template <class T>
cudaError_t launch_pack_full(const double* src, T* dst, int nxe, int nye, int pitch, cudaStream_t st) {
    k_pack_full<T><<<dim3((nxe + 255) / 256, nye), 256, 0, st>>>(src, dst, nxe, pitch);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_nest_ring(const Grid<T>& f, const Ctl* fctl, const Grid<T>& c, const Ctl* cctl, int ix0, int iy0,
                             double w, double eps, cudaStream_t st) {
    const long long n = 2LL * PAD * (f.nx + 2 * PAD) + 2LL * PAD * f.ny;
    k_nest_ring<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, fctl, c, cctl, ix0, iy0, w, eps);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_ring_outflow(const Grid<T>& g, const Ctl* ctl, cudaStream_t st) {
    const long long n = 2LL * PAD * (g.nx + 2 * PAD) + 2LL * PAD * g.ny;
    k_ring_outflow<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, ctl);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_nest_restrict(const Grid<T>& f, const Ctl* fctl, const Grid<T>& c, const Ctl* cctl, int ix0, int iy0,
                                 cudaStream_t st) {
    const int n = (f.nx / 4) * (f.ny / 4);
    k_nest_restrict<T><<<(n + 255) / 256, 256, 0, st>>>(f, fctl, c, cctl, ix0, iy0);
    return cudaGetLastError();
}

template <class T>
__global__ void k_unpack(const T* __restrict__ src, double* __restrict__ dst, int nx, int ny, int pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i < nx) dst[(size_t)j * nx + i] = (double)src[(size_t)(j + PAD) * pitch + (i + PAD)];
}

// Bed of the padded layout: walls outside the interior, 0 inside.
template <class T>
__global__ void k_fill_bed(T* b, int nx, int ny, int pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= pitch) return;
    const bool inside = i >= PAD && i < nx + PAD && j >= PAD && j < ny + PAD;
    b[(size_t)j * pitch + i] = inside ? T(0) : T(WALL_BED);
}

template <class T>
cudaError_t launch_fill_bed(T* b, int nx, int ny, int pitch, cudaStream_t st) {
    k_fill_bed<T><<<dim3((pitch + 255) / 256, ny + 2 * PAD), 256, 0, st>>>(b, nx, ny, pitch);
    return cudaGetLastError();
}

template <class T>
__global__ void k_scatter(T* dst, const int* idx, const double* val, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) dst[idx[m]] = (T)val[m];
}

template <class T>
cudaError_t launch_pack(const double* src, T* dst, int nx, int ny, int pitch, cudaStream_t st, unsigned* flag,
                        int check_neg) {
    k_pack<T><<<dim3((nx + 255) / 256, ny), 256, 0, st>>>(src, dst, nx, ny, pitch, flag, check_neg);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_unpack(const T* src, double* dst, int nx, int ny, int pitch, cudaStream_t st) {
    k_unpack<T><<<dim3((nx + 255) / 256, ny), 256, 0, st>>>(src, dst, nx, ny, pitch);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_scatter(T* dst, const int* idx, const double* val, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_scatter<T><<<(n + 127) / 128, 128, 0, st>>>(dst, idx, val, n);
    return cudaGetLastError();
}

#define SWE_INSTANTIATE(T)                                                                           \
    template cudaError_t launch_fused<T>(const FusedArgs<T>&, cudaStream_t);                         \
    template cudaError_t prepare_fused<T>(int*);                                                     \
    template cudaError_t prepare_fused_batch<T>(int*);                                               \
    template cudaError_t launch_fused_batch<T>(const BatchArgs<T>&, int, cudaStream_t);              \
    template cudaError_t launch_staged<T>(const StagedArgs<T>&, cudaStream_t);                       \
    template cudaError_t launch_state_speed<T>(const StagedArgs<T>&, cudaStream_t, int);                  \
    template cudaError_t launch_state_speed_region<T>(const StagedArgs<T>&, int, int, int, int, cudaStream_t); \
    template cudaError_t launch_pack<T>(const double*, T*, int, int, int, cudaStream_t, unsigned*, int); \
    template cudaError_t launch_band_acc<T>(const StagedArgs<T>&, cudaStream_t);                     \
    template cudaError_t launch_unpack<T>(const T*, double*, int, int, int, cudaStream_t);           \
    template cudaError_t launch_scatter<T>(T*, const int*, const double*, int, cudaStream_t);        \
    template cudaError_t launch_fill_bed<T>(T*, int, int, int, cudaStream_t);                        \
    template cudaError_t launch_pack_full<T>(const double*, T*, int, int, int, cudaStream_t);       \
    template cudaError_t launch_nest_ring<T>(const Grid<T>&, const Ctl*, const Grid<T>&, const Ctl*, int, int, \
                                             double, double, cudaStream_t);                         \
    template cudaError_t launch_ring_outflow<T>(const Grid<T>&, const Ctl*, cudaStream_t);         \
    template cudaError_t launch_nest_restrict<T>(const Grid<T>&, const Ctl*, const Grid<T>&, const Ctl*, int, \
                                                 int, cudaStream_t);                                \
    template size_t fused_smem_bytes<T>();

}  // namespace swe
