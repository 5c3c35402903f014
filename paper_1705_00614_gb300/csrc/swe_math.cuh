// Per-cell and per-face arithmetic of one CSPH-TVD time step (Sec. 2.3,
// Fig. 2; kernels K2-K8 of Sec. 3), templated on the arithmetic type.
//
// Every function takes values, not pointers, so the fused streaming kernel
// (shared-memory rings) and the staged kernels (one kernel per stage, global
// memory) run the same instructions.  The operation order of each formula is
// fixed and is the one of the scheme's written definition, so the FP64
// instantiation (compiled without FMA contraction) rounds like a plain
// sequential evaluation of the same formulas, with one deliberate exception:
// face depths eta - b* are formed as H + (b - b*) (see face_delta), which
// differs from evaluating eta first by one rounding of eta.  The FP32
// instantiation multiplies by reciprocals instead of dividing (one reciprocal
// shared by the two components of a vector, and host-computed constants such
// as -g / (4 h)); its accuracy is set against the FP64 oracle, not against a
// sequential FP32 evaluation.
//
// Walls: the device layout surrounds every grid by a ring of cells whose bed
// is WALL_BED (1e30) and whose depth is 0, and a closed gate is a cell whose
// bed is WALL_BED.  With that bed every face formula below yields exactly the
// value of a reflective wall (no pressure difference, no flux, no viscous
// stress), so no kernel needs a boundary branch.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace swe {

constexpr double WALL_BED = 1.0e30;
constexpr double WALL_TEST = 1.0e29;  // beds at or above this are walls

template <class T>
struct Phys {
    T g;     // gravity
    T h;     // cell size dx = dy
    T eps;   // dry threshold
    T nu;    // viscosity
    T f;     // Coriolis parameter
    T wx, wy;  // wind
    T ca, ra;  // C_a and rho_a / rho
    // distributed sources of Eq. 1 on every non-wall cell: rain r and the
    // losses e + i (evaporation, infiltration); dist = any of them nonzero
    T rain, loss;
    int dist;
    // derived constants for the FP32 forms, which multiply by reciprocals
    // (the fast-math build turns every division into one anyway):
    // -g / (4 h), nu / h^2, C_a rho_a / rho, 1 / g, 1 / h (phys_derive)
    T gq, cv, cara, ig, ih;
};

template <class T>
__host__ __device__ inline void phys_derive(Phys<T>& P) {
    P.gq = -P.g / (T(4) * P.h);
    P.cv = P.nu / (P.h * P.h);
    P.cara = P.ca * P.ra;
    P.ig = T(1) / P.g;
    P.ih = T(1) / P.h;
}

// Packed FP32 pairs: on sm_100 and later one add / mul / fma instruction
// works on two FP32 lanes of a 64-bit register pair.  The FP32 instantiation
// uses them for the x and y components of its vectors (velocities,
// accelerations, momenta, pairs of faces), which halves the issue slots of
// that arithmetic.  Each lane rounds like the scalar FP32 operation of the
// fast-math build (round to nearest, denormals flushed to zero); an explicit
// mul2 is never contracted with a following add.
struct f2 {
    float x, y;
};
__device__ __forceinline__ f2 mk2(float x, float y) { return f2{x, y}; }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.ftz.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.ftz.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.ftz.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// a * b + c
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("{\n\t.reg .b64 pa, pb, pc, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%6, %7};\n\tfma.rn.ftz.f32x2 pr, pa, pb, pc;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ f2 max02(f2 a) { return f2{fmaxf(0.f, a.x), fmaxf(0.f, a.y)}; }
__device__ __forceinline__ f2 sel2(bool c, f2 a) { return f2{c ? a.x : 0.f, c ? a.y : 0.f}; }

// q = a / d and r = b / d; FP32 shares one reciprocal, FP64 divides (the
// oracle's rounding)
template <class T>
__device__ __forceinline__ void div2(T a, T b, T d, T& q, T& r) {
    if constexpr (sizeof(T) == 4) {
        const T id = T(1) / d;
        const f2 v = mul2(mk2(a, b), mk2(id, id));
        q = v.x;
        r = v.y;
    } else {
        q = a / d;
        r = b / d;
    }
}

// div2 where cond holds, else q = r = 0.  FP32 evaluates on every lane and
// selects (cheaper than diverging); FP64, whose divisions are long sequences
// on a slow pipe, divides only where cond holds.  Same values either way.
template <class T>
__device__ __forceinline__ void div2_if(bool cond, T a, T b, T d, T& q, T& r) {
    if constexpr (sizeof(T) == 4) {
        div2(a, b, d, q, r);
        q = cond ? q : T(0);
        r = cond ? r : T(0);
    } else {
        q = T(0);
        r = T(0);
        if (cond) div2(a, b, d, q, r);
    }
}


// (u + s a) / d for the two components of a vector (the implicit-friction
// velocity updates of the predictor and the corrector)
template <class T>
__device__ __forceinline__ void lin_div2(T ux, T uy, T s, T ax, T ay, T d, T& qx, T& qy) {
    if constexpr (sizeof(T) == 4) {
        const f2 v = fma2(mk2(s, s), mk2(ax, ay), mk2(ux, uy));
        div2(v.x, v.y, d, qx, qy);
    } else {
        div2(ux + s * ax, uy + s * ay, d, qx, qy);
    }
}

// Multiplications whose products must cancel exactly (h_R^2 - h_L^2 with
// h_R == h_L at rest) are kept out of FMA contraction.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <class T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <class T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <class T> __device__ __forceinline__ T tsgn(T a) { return a > T(0) ? T(1) : (a < T(0) ? T(-1) : T(0)); }

// H^{4/3} in FP64: H * cbrt(H).  The FP32 friction takes H^{-4/3} as
// 2^{-(4/3) log2 H} instead (two SFU operations in the fast-math build;
// relative error ~2e-7).
__device__ __forceinline__ double pow43(double x) { return x * cbrt(x); }

template <class T>
__device__ __forceinline__ bool is_wet(T H, T b, T eps) { return H > eps && b < T(WALL_TEST); }

// infinite or NaN, tested on the exponent bits (integer work)
__device__ __forceinline__ bool nonfinite_bits(float x) {
    return (__float_as_uint(x) & 0x7F800000u) == 0x7F800000u;
}
__device__ __forceinline__ bool nonfinite_bits(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7FF0000000000000ull) == 0x7FF0000000000000ull;
}

__device__ __forceinline__ bool is_neg_zero(float x) { return __float_as_uint(x) == 0x80000000u; }
__device__ __forceinline__ bool is_neg_zero(double x) {
    return (unsigned long long)__double_as_longlong(x) == 0x8000000000000000ull;
}

// Hydrostatic reconstruction at the face between L and R (Audusse et al.):
// b* = max(b_L, b_R), h_{L,R} = max(0, eta_{L,R} - b*); returns h_R^2 - h_L^2.
// eta - b* is evaluated as H + (b - b*): the bed difference is exact or
// nearly so, and a thin layer over high terrain keeps its relative
// precision instead of cancelling in eta = H + b (which in FP32 has an
// absolute resolution of ~2e-6 m at 30 m).  A face with a wall is closed.
template <class T>
__device__ __forceinline__ T face_delta(T hsL, T bL, T hsR, T bR) {
    T bs = tmax(bL, bR);
    if (bs >= T(WALL_TEST)) return T(0);
    T hl = tmax(T(0), hsL + (bL - bs));
    T hr = tmax(T(0), hsR + (bR - bs));
    return mul_rn(hr, hr) - mul_rn(hl, hl);
}

// One neighbour as seen by the force evaluation.
template <class T>
struct Nb {
    T hs, b, ux, uy;
    bool wet;
};

// Accelerations of Eqs. 2-4 on a wet cell without friction (stage I, K2;
// and K5 at t_{n+1/2}): a = a^P + a^V + a^C + a^W.
template <class T>
__device__ __forceinline__ void accel(const Phys<T>& P, T hs, T b, T ux, T uy, const Nb<T>& W,
                                      const Nb<T>& E, const Nb<T>& S, const Nb<T>& N, T& ax, T& ay) {
    if constexpr (sizeof(T) == 4) {
        // The same terms on (x, y) pairs.  Faces W and S (the cell on their
        // right / upper side) and faces E and N (the cell on their left /
        // lower side) are each evaluated as one pair of face_delta.
        const f2 bsm = mk2(fmaxf(W.b, b), fmaxf(S.b, b));
        const f2 bsp = mk2(fmaxf(b, E.b), fmaxf(b, N.b));
        const f2 self = mk2(hs, hs), bb = mk2(b, b);
        const f2 hlm = max02(add2(mk2(W.hs, S.hs), sub2(mk2(W.b, S.b), bsm)));
        const f2 hrm = max02(add2(self, sub2(bb, bsm)));
        const f2 hlp = max02(add2(self, sub2(bb, bsp)));
        const f2 hrp = max02(add2(mk2(E.hs, N.hs), sub2(mk2(E.b, N.b), bsp)));
        // h_R^2 - h_L^2 as (h_R - h_L)(h_R + h_L): exactly zero when
        // h_R == h_L (still water) even where the assembler fuses the
        // product into a following add (a difference of two rounded
        // squares would then keep one square's rounding error)
        f2 dm = mul2(sub2(hrm, hlm), add2(hrm, hlm));
        f2 dp = mul2(sub2(hrp, hlp), add2(hrp, hlp));
        dm.x = bsm.x >= T(WALL_TEST) ? T(0) : dm.x;
        dm.y = bsm.y >= T(WALL_TEST) ? T(0) : dm.y;
        dp.x = bsp.x >= T(WALL_TEST) ? T(0) : dp.x;
        dp.y = bsp.y >= T(WALL_TEST) ? T(0) : dp.y;
        const T ih = T(1) / hs;
        const T coef = P.gq * ih;
        const f2 u = mk2(ux, uy);
        // viscosity: no stress from non-wet neighbours
        f2 l = sel2(W.wet, sub2(mk2(W.ux, W.uy), u));
        l = add2(l, sel2(E.wet, sub2(mk2(E.ux, E.uy), u)));
        l = add2(l, sel2(S.wet, sub2(mk2(S.ux, S.uy), u)));
        l = add2(l, sel2(N.wet, sub2(mk2(N.ux, N.uy), u)));
        // wind stress
        const f2 dw = sub2(mk2(P.wx, P.wy), u);
        const T wm = sqrtf(dw.x * dw.x + dw.y * dw.y);
        const T cw = P.cara * wm * ih;
        // a = a^P + a^V + a^C + a^W
        f2 a = mul2(mk2(coef, coef), add2(dm, dp));
        a = fma2(mk2(P.cv, P.cv), l, a);
        a = fma2(mk2(P.f, -P.f), mk2(uy, ux), a);
        a = fma2(mk2(cw, cw), dw, a);
        ax = a.x;
        ay = a.y;
        return;
    }
    // pressure -g grad(eta) in the well-balanced face form
    T dxm = face_delta(W.hs, W.b, hs, b);
    T dxp = face_delta(hs, b, E.hs, E.b);
    T dym = face_delta(S.hs, S.b, hs, b);
    T dyp = face_delta(hs, b, N.hs, N.b);
    T coef, ih = T(0);
    if constexpr (sizeof(T) == 4) {
        ih = T(1) / hs;
        coef = P.gq * ih;
    } else {
        coef = -P.g / (T(4) * P.h * hs);
    }
    T aPx = coef * (dxm + dxp);
    T aPy = coef * (dym + dyp);
    // viscosity: W, E, S, N; no stress from non-wet neighbours
    T lx = T(0), ly = T(0);
    lx = lx + (W.wet ? W.ux - ux : T(0)); ly = ly + (W.wet ? W.uy - uy : T(0));
    lx = lx + (E.wet ? E.ux - ux : T(0)); ly = ly + (E.wet ? E.uy - uy : T(0));
    lx = lx + (S.wet ? S.ux - ux : T(0)); ly = ly + (S.wet ? S.uy - uy : T(0));
    lx = lx + (N.wet ? N.ux - ux : T(0)); ly = ly + (N.wet ? N.uy - uy : T(0));
    T cv;
    if constexpr (sizeof(T) == 4) cv = P.cv;
    else cv = P.nu / (P.h * P.h);
    T aVx = cv * lx, aVy = cv * ly;
    // Coriolis 2 U x Omega
    T aCx = P.f * uy, aCy = -P.f * ux;
    // wind stress
    T dwx = P.wx - ux, dwy = P.wy - uy;
    T wm = sqrt(dwx * dwx + dwy * dwy);
    T cw;
    if constexpr (sizeof(T) == 4) cw = P.cara * wm * ih;
    else cw = P.ca * P.ra * wm / hs;
    T aWx = cw * dwx, aWy = cw * dwy;
    ax = ((aPx + aVx) + aCx) + aWx;
    ay = ((aPy + aVy) + aCy) + aWy;
}

// Manning friction coefficient of a wet cell: F^fric = -phi U with
// phi = g n^2 |U| / H^{4/3} (Eq. 4); it depends on the cell alone.
template <class T>
__device__ __forceinline__ T friction(const Phys<T>& P, T hs, T nm, T ux, T uy) {
    T um = sqrt(ux * ux + uy * uy);
    if constexpr (sizeof(T) == 4) return P.g * nm * nm * um * exp2f(-1.33333333f * log2f(hs));
    else return P.g * nm * nm * um / pow43(hs);
}

// Forces of Eqs. 2-4 on a wet cell: the accelerations and the friction
// coefficient.
template <class T>
__device__ __forceinline__ void forces(const Phys<T>& P, T hs, T b, T nm, T ux, T uy,
                                       const Nb<T>& W, const Nb<T>& E, const Nb<T>& S,
                                       const Nb<T>& N, T& ax, T& ay, T& phi) {
    accel(P, hs, b, ux, uy, W, E, S, N, ax, ay);
    phi = friction(P, hs, nm, ux, uy);
}

// Signal speed of a wet cell (Fig. 2): max(U_s, U_p).
template <class T>
__device__ __forceinline__ T cell_speed(const Phys<T>& P, T H, T ux, T uy, T ax, T ay) {
    T c = sqrt(P.g * H);
    T us = tmax(fabs(ux), fabs(uy)) + c;
    T upx, upy;
    if constexpr (sizeof(T) == 4) {
        // sgn(a) sqrt(h |a|) as a sign transfer (the same value)
        const f2 ha = mul2(mk2(P.h, P.h), mk2(fabsf(ax), fabsf(ay)));
        const f2 up = add2(mk2(ux, uy), mk2(copysignf(sqrtf(ha.x), ax), copysignf(sqrtf(ha.y), ay)));
        upx = fabsf(up.x);
        upy = fabsf(up.y);
    } else {
        upx = fabs(ux + tsgn(ax) * sqrt(P.h * fabs(ax)));
        upy = fabs(uy + tsgn(ay) * sqrt(P.h * fabs(ay)));
    }
    return tmax(us, tmax(upx, upy));
}

template <class T>
__device__ __forceinline__ T minmod(T a, T b) {
    if constexpr (sizeof(T) == 4) {
        // the same value without branches (a zero result may carry a's sign):
        // the smaller magnitude when both have one sign, else zero
        const float m = fminf(fabsf(a), fabsf(b));
        return ((__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u) ? 0.0f : copysignf(m, a);
    }
    if (a > T(0) && b > T(0)) return a < b ? a : b;
    if (a < T(0) && b < T(0)) return a > b ? a : b;
    return T(0);
}

// Two-rarefaction approximate Riemann solution (Toro 2001) sampled at
// x/t = 0; a side with depth <= eps is dry (dry-bed fan).
template <class T>
__device__ __forceinline__ void riemann(T g, T ig, T eps, T hl, T ul, T hr, T ur, T& h, T& u) {
    // c^2 / g: FP32 multiplies by 1/g
    auto c2g = [&](T c) -> T {
        if constexpr (sizeof(T) == 4) return c * c * ig;
        else return c * c / g;
    };
    bool dl = !(hl > eps), dr = !(hr > eps);
    h = T(0);
    u = T(0);
    if (dl && dr) return;
    T cl = dl ? T(0) : sqrt(g * hl);
    T cr = dr ? T(0) : sqrt(g * hr);
    if (dr) {
        if (ul - cl >= T(0)) { h = hl; u = ul; }
        else if (ul + T(2) * cl > T(0)) { T c = (ul + T(2) * cl) / T(3); h = c2g(c); u = c; }
    } else if (dl) {
        if (ur + cr <= T(0)) { h = hr; u = ur; }
        else if (ur - T(2) * cr < T(0)) { T c = (T(2) * cr - ur) / T(3); h = c2g(c); u = -c; }
    } else if (T(2) * (cl + cr) <= ur - ul) {
        if (ul - cl >= T(0)) { h = hl; u = ul; }
        else if (ul + T(2) * cl > T(0)) { T c = (ul + T(2) * cl) / T(3); h = c2g(c); u = c; }
        else if (ur + cr <= T(0)) { h = hr; u = ur; }
        else if (ur - T(2) * cr < T(0)) { T c = (T(2) * cr - ur) / T(3); h = c2g(c); u = -c; }
    } else {
        T us = T(0.5) * (ul + ur) + cl - cr;
        T cs = T(0.5) * (cl + cr) + T(0.25) * (ul - ur);
        if (us >= T(0)) {
            if (ul - cl >= T(0)) { h = hl; u = ul; }
            else if (us - cs >= T(0)) { T c = (ul + T(2) * cl) / T(3); h = c2g(c); u = c; }
            else { h = c2g(cs); u = us; }
        } else {
            if (ur + cr <= T(0)) { h = hr; u = ur; }
            else if (us + cs <= T(0)) { T c = (T(2) * cr - ur) / T(3); h = c2g(c); u = -c; }
            else { h = c2g(cs); u = us; }
        }
    }
}

// Eulerian cell values (after the Lagrangian stage) used by the face fluxes:
// w = (H~, U^x, U^y, U~'x, U~'y), the bed, and whether the cell is wet.  The
// free surface eta~ = H~ + b is reconstructed through its differences
// (H~ and b differenced separately), never formed directly.
template <class T>
struct ECell {
    T w[5];
    T b;
    bool wt;
};

// MUSCL slope of one cell along the face normal (minmod; zero unless the
// cell and both neighbours along the normal are wet).
template <class T>
__device__ __forceinline__ void slopes(const ECell<T>& m, const ECell<T>& c, const ECell<T>& p, T s[5]) {
    bool lim = m.wt && c.wt && p.wt;
    if constexpr (sizeof(T) == 4) {
        // differences on pairs: (H~, b) and the velocity pairs
        const f2 dm0 = sub2(mk2(c.w[0], c.b), mk2(m.w[0], m.b)), dp0 = sub2(mk2(p.w[0], p.b), mk2(c.w[0], c.b));
        s[0] = lim ? minmod(dm0.x + dm0.y, dp0.x + dp0.y) : T(0);
#pragma unroll
        for (int q = 1; q < 5; q += 2) {
            const f2 dm = sub2(mk2(c.w[q], c.w[q + 1]), mk2(m.w[q], m.w[q + 1]));
            const f2 dp = sub2(mk2(p.w[q], p.w[q + 1]), mk2(c.w[q], c.w[q + 1]));
            s[q] = lim ? minmod(dm.x, dp.x) : T(0);
            s[q + 1] = lim ? minmod(dm.y, dp.y) : T(0);
        }
        return;
    }
    s[0] = lim ? minmod((c.w[0] - m.w[0]) + (c.b - m.b), (p.w[0] - c.w[0]) + (p.b - c.b)) : T(0);
#pragma unroll
    for (int q = 1; q < 5; ++q) s[q] = lim ? minmod(c.w[q] - m.w[q], p.w[q] - c.w[q]) : T(0);
}

// Flux through the face between L and R (stage III, K7) given the cells'
// slopes along the normal; nq = 1 for x faces (normal velocity U^x), 2 for
// y faces.  Mass flux F_H = h u of the sampled Riemann state; momentum flux
// F_H times the upwind reconstructed U~'.
template <class T>
__device__ __forceinline__ void face_flux(const Phys<T>& P, const ECell<T>& L, const T sL[5],
                                          const ECell<T>& R, const T sR[5], int nq, T& FH,
                                          T& FQx, T& FQy) {
    T wl[5], wr[5];
    if constexpr (sizeof(T) == 4) {
        // the face values this face uses, as (left, right) pairs: surface,
        // normal velocity (nq), and the two upwind momentum velocities; the
        // tangential mean velocity is not reconstructed (unused, so its
        // slope is never formed either)
        const f2 lr = mk2(0.5f, -0.5f);
        const f2 d0 = fma2(lr, mk2(sL[0], sR[0]), mk2(L.w[0], R.w[0]));
        const f2 dn = fma2(lr, mk2(sL[nq], sR[nq]), mk2(L.w[nq], R.w[nq]));
        const f2 l2 = fma2(mk2(0.5f, 0.5f), mk2(sL[3], sL[4]), mk2(L.w[3], L.w[4]));
        const f2 r2 = fma2(mk2(-0.5f, -0.5f), mk2(sR[3], sR[4]), mk2(R.w[3], R.w[4]));
        wl[0] = d0.x;
        wr[0] = d0.y;
        wl[1] = wl[2] = dn.x;
        wr[1] = wr[2] = dn.y;
        wl[3] = l2.x;
        wl[4] = l2.y;
        wr[3] = r2.x;
        wr[4] = r2.y;
    } else {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            wl[q] = L.w[q] + T(0.5) * sL[q];
            wr[q] = R.w[q] - T(0.5) * sR[q];
        }
    }
    T bs = tmax(L.b, R.b);
    FH = T(0);
    FQx = T(0);
    FQy = T(0);
    if (bs >= T(WALL_TEST)) return;
    // eta~ at the face minus b*: (H~ + half slope) + (b - b*)
    T hl, hr;
    if constexpr (sizeof(T) == 4) {
        const f2 h2 = max02(add2(mk2(wl[0], wr[0]), sub2(mk2(L.b, R.b), mk2(bs, bs))));
        hl = h2.x;
        hr = h2.y;
    } else {
        hl = tmax(T(0), wl[0] + (L.b - bs));
        hr = tmax(T(0), wr[0] + (R.b - bs));
    }
    T un_l = nq == 1 ? wl[1] : wl[2];
    T un_r = nq == 1 ? wr[1] : wr[2];
    T hs, us;
    riemann(P.g, P.ig, P.eps, hl, un_l, hr, un_r, hs, us);
    FH = hs * us;
    if constexpr (sizeof(T) == 4) {
        const bool up = FH >= T(0);
        const f2 fq = mul2(mk2(FH, FH), mk2(up ? wl[3] : wr[3], up ? wl[4] : wr[4]));
        FQx = fq.x;
        FQy = fq.y;
    } else {
        FQx = FH * (FH >= T(0) ? wl[3] : wr[3]);
        FQy = FH * (FH >= T(0) ? wl[4] : wr[4]);
    }
}

// Point source of Eqs. 1-3 on the post-Lagrangian state (ts = tau sigma):
// H~ = max(0, H + ts).  Inflow (sigma > 0) brings water with the source
// velocity V; a drain takes water with the cell's velocity U~ and never more
// than the cell holds, so a drain that empties the cell (H + ts <= 0) leaves
// it without momentum.
template <class T>
__device__ __forceinline__ void point_source(T H, T sig, T ts, T vx, T vy, T utx, T uty, T& ht, T& qtx, T& qty) {
    const T hp = H + ts;
    ht = tmax(T(0), hp);
    const bool keep = sig > T(0) || hp > T(0);
    if constexpr (sizeof(T) == 4) {
        const bool in = sig > T(0);
        const f2 q = fma2(mk2(ts, ts), mk2(in ? vx : utx, in ? vy : uty), mul2(mk2(H, H), mk2(utx, uty)));
        qtx = keep ? q.x : T(0);
        qty = keep ? q.y : T(0);
    } else {
        qtx = keep ? H * utx + (sig > T(0) ? ts * vx : ts * utx) : T(0);
        qty = keep ? H * uty + (sig > T(0) ? ts * vy : ts * uty) : T(0);
    }
}

// Rain, evaporation and infiltration (Eq. 1 sigma) on a non-wall cell after
// the point sources (hp = H + tau sigma_pt): depth
// H~ = max(0, hp + tau (r - e - i)); rain brings water at rest, the losses
// take water with its velocity U~, at most the depth max(0, hp) the point
// source left.
template <class T>
__device__ __forceinline__ void distributed_sources(const Phys<T>& P, T tau, T hp, T utx, T uty, T& ht, T& qtx,
                                                    T& qty) {
    const T taken = tmin(tau * P.loss, tmax(T(0), hp));
    ht = tmax(T(0), hp + tau * (P.rain - P.loss));
    qtx = qtx - taken * utx;
    qty = qty - taken * uty;
}

// Hydrograph value q(t) of one row (kind, peak, t_p, s), in FP64.
__device__ __forceinline__ double hydro_value(const double* row, double t) {
    if (row[0] == 0.0) {
        double z = (t - row[2]) / row[3];
        return row[1] * exp(-0.5 * z * z);
    }
    return row[1];
}

}  // namespace swe
