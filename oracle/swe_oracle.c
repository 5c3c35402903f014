/*
 * FP64 CPU oracle of one CSPH-TVD shallow-water time step.
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plain reference that the CUDA
 * library is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never does.
 * It shares no code, header or constant with the CUDA path.
 *
 * Every stage is one plain loop nest over the whole grid, in the order of
 * the paper's scheme (Sec. 2.3, Fig. 2; kernel list K2-K8 of Sec. 3):
 *   1. primitives U = HU/H                                  (Eqs. 1-3)
 *   2. forces at t_n: pressure from the free-surface gradient of eta = H + b,
 *      viscosity, Coriolis, wind, Manning friction        (Eqs. 2-4, K2)
 *   3. time step tau_n from U_s and U_p with Courant number K   (Fig. 2, K3)
 *   4. Lagrangian predictor U*, H* at t_{n+1/2}            (Sec. 2.3, K4)
 *   5. forces at t_{n+1/2}, Lagrangian corrector, sources  (K5, K6)
 *   6. Eulerian face fluxes from an approximate Riemann solution (K7)
 *   7. final update, particles back to cell centres        (K8)
 * Fig. 2 is missing from the available text, so the formulas of each stage
 * are a documented reading of the paper built from named published pieces:
 * hydrostatic reconstruction (Audusse et al. 2004), surface-gradient (eta)
 * reconstruction with the minmod limiter (van Leer MUSCL), and the
 * two-rarefaction approximate Riemann solver (Toro 2001).
 *
 * Conventions: arrays are row-major [ny][nx], index k = j*nx + i, x along i.
 * A cell is wet when it is not solid and its depth exceeds eps.  Cells
 * outside the grid and solid (closed-gate) cells are walls: never wet, no
 * face flux, and no hydrostatic pressure difference across their faces.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, IEEE
 * round-to-nearest), so every operation is a correctly rounded FP64 op
 * except the libm calls sqrt (exact), cbrt and exp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny;
    double dx;      /* h = dx = dy (Sec. 2.2) */
    double g;       /* gravitational acceleration */
    double cfl;     /* Courant number K, 0 < K < 1 (Fig. 2) */
    double eps;     /* dry threshold (the Eps of K8) */
    double dt_max;  /* upper bound of tau */
    double dt_fixed;/* > 0: tau forced to this value */
    double t_end;   /* > 0: tau clamped so that t never passes t_end */
    double nu;      /* turbulent viscosity (Eq. 4) */
    double f;       /* Coriolis parameter 2 Omega sin(phi) (Eq. 4) */
    double wx, wy;  /* wind velocity W (Eq. 4) */
    double ca;      /* C_a (Eq. 4) */
    double ra;      /* rho_a / rho (Eq. 4) */
    double rain;    /* distributed sources of Eq. 1 (m/s, every non-wall */
    double evap;    /*   cell): rainfall adds water without momentum; */
    double infil;   /*   evaporation and infiltration take water with its velocity */
} orc_params;

typedef struct {
    int32_t n;
    const int32_t *ix, *iy, *hydro;
    const double *weight, *vx, *vy;
    int32_t nh;
    const double *hydro_tab; /* nh rows of (kind, peak, tp, s) */
} orc_sources;

/* Optional per-stage outputs (any pointer may be NULL). */
typedef struct {
    double *ux, *uy;          /* U at t_n */
    double *ax, *ay, *phi;    /* accelerations and friction coefficient at t_n */
    double *usx, *usy, *hs;   /* predictor U*, H* (t_{n+1/2}) */
    double *ax2, *ay2, *phi2; /* accelerations at t_{n+1/2} */
    double *utx, *uty;        /* corrector velocity U~ (t_{n+1}) */
    double *uhx, *uhy;        /* mean velocity U^ = (U + U~)/2 */
    double *ht, *qtx, *qty;   /* post-Lagrangian H~, Q~ (the paper's Ht, HVt) */
    double *upx, *upy;        /* U~' = Q~/H~ */
    double *fx;               /* [3][ny][nx+1] x-face fluxes (F_H, F_Qx, F_Qy) */
    double *fy;               /* [3][ny+1][nx] y-face fluxes */
} orc_stages;

typedef struct {
    double tau, t_new, smax, mass, clip_vol, src_vol;
    int64_t wet;
} orc_info;

#define IX(i, j) ((size_t)(j) * (size_t)nx + (size_t)(i))

static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }
static double sgn(double a) { return a > 0.0 ? 1.0 : (a < 0.0 ? -1.0 : 0.0); }

/* Hydrostatic reconstruction at the face between cells L and R (Audusse et
 * al. 2004): with b* = max(b_L, b_R), h_L = max(0, eta_L - b*),
 * h_R = max(0, eta_R - b*), return h_R^2 - h_L^2.  The pressure force the
 * face puts on its left cell is (g/2) H_L^2 + (g/4)(h_R^2 - h_L^2), and on
 * its right cell (g/2) H_R^2 - (g/4)(h_R^2 - h_L^2).  Walls give 0. */
static double face_delta(double hsL, double bL, int wallL, double hsR, double bR, int wallR)
{
    if (wallL || wallR) return 0.0;
    double etaL = hsL + bL, etaR = hsR + bR;
    double bs = dmax(bL, bR);
    double hl = dmax(0.0, etaL - bs);
    double hr = dmax(0.0, etaR - bs);
    return hr * hr - hl * hl;
}

/* Forces of Eqs. 2-4 on every wet cell, from depth hs and velocity (ux, uy):
 *   a^P: -(g / (4 h Hs)) (Delta_{i-1/2} + Delta_{i+1/2}) per direction, the
 *        hydrostatic-reconstruction form of -g grad(eta) (well balanced:
 *        zero when eta is flat);
 *   a^V: nu * 5-point Laplacian of U, a non-wet neighbour counted as equal
 *        to the cell (no stress across dry or wall faces);
 *   a^C: 2 U x Omega = f (U_y, -U_x);
 *   a^W: C_a (rho_a/rho) (W - U)|W - U| / Hs;
 *   phi: friction coefficient g n_M^2 |U| / Hs^{4/3}, so that
 *        F^fric = -(lambda/2) U|U| = -phi U with lambda = 2 g n_M^2 / H^{4/3}.
 * Non-wet cells get zero. */
static void forces(const orc_params* p, const double* hs, const double* ux, const double* uy,
                   const unsigned char* wet, const unsigned char* solid, const double* b,
                   const double* nm, double* ax, double* ay, double* phi)
{
    const int nx = p->nx, ny = p->ny;
    const double h = p->dx, g = p->g;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t k = IX(i, j);
            if (!wet[k]) { ax[k] = 0.0; ay[k] = 0.0; phi[k] = 0.0; continue; }
            /* pressure through the four faces */
            double dxm = (i > 0) ? face_delta(hs[k - 1], b[k - 1], solid[k - 1], hs[k], b[k], solid[k]) : 0.0;
            double dxp = (i < nx - 1) ? face_delta(hs[k], b[k], solid[k], hs[k + 1], b[k + 1], solid[k + 1]) : 0.0;
            double dym = (j > 0) ? face_delta(hs[k - nx], b[k - nx], solid[k - nx], hs[k], b[k], solid[k]) : 0.0;
            double dyp = (j < ny - 1) ? face_delta(hs[k], b[k], solid[k], hs[k + nx], b[k + nx], solid[k + nx]) : 0.0;
            double coef = -g / (4.0 * h * hs[k]);
            double aPx = coef * (dxm + dxp);
            double aPy = coef * (dym + dyp);
            /* viscosity: neighbours W, E, S, N */
            double lx = 0.0, ly = 0.0, dvx, dvy;
            dvx = (i > 0 && wet[k - 1]) ? ux[k - 1] - ux[k] : 0.0;
            dvy = (i > 0 && wet[k - 1]) ? uy[k - 1] - uy[k] : 0.0;
            lx = lx + dvx; ly = ly + dvy;
            dvx = (i < nx - 1 && wet[k + 1]) ? ux[k + 1] - ux[k] : 0.0;
            dvy = (i < nx - 1 && wet[k + 1]) ? uy[k + 1] - uy[k] : 0.0;
            lx = lx + dvx; ly = ly + dvy;
            dvx = (j > 0 && wet[k - nx]) ? ux[k - nx] - ux[k] : 0.0;
            dvy = (j > 0 && wet[k - nx]) ? uy[k - nx] - uy[k] : 0.0;
            lx = lx + dvx; ly = ly + dvy;
            dvx = (j < ny - 1 && wet[k + nx]) ? ux[k + nx] - ux[k] : 0.0;
            dvy = (j < ny - 1 && wet[k + nx]) ? uy[k + nx] - uy[k] : 0.0;
            lx = lx + dvx; ly = ly + dvy;
            double cv = p->nu / (h * h);
            double aVx = cv * lx, aVy = cv * ly;
            /* Coriolis */
            double aCx = p->f * uy[k], aCy = -p->f * ux[k];
            /* wind */
            double dwx = p->wx - ux[k], dwy = p->wy - uy[k];
            double wm = sqrt(dwx * dwx + dwy * dwy);
            double cw = p->ca * p->ra * wm / hs[k];
            double aWx = cw * dwx, aWy = cw * dwy;
            ax[k] = ((aPx + aVx) + aCx) + aWx;
            ay[k] = ((aPy + aVy) + aCy) + aWy;
            /* Manning friction coefficient */
            double um = sqrt(ux[k] * ux[k] + uy[k] * uy[k]);
            phi[k] = g * nm[k] * nm[k] * um / (hs[k] * cbrt(hs[k]));
        }
    }
}

/* Largest signal speed over wet cells (Fig. 2):
 *   U_s = max(|U_x|, |U_y|) + sqrt(g H)
 *   U_p = max(|U_x + sgn(a_x) sqrt(h |a_x|)|, |U_y + sgn(a_y) sqrt(h |a_y|)|). */
static double max_speed(const orc_params* p, const double* H, const double* ux, const double* uy,
                        const double* ax, const double* ay, const unsigned char* wet)
{
    const int nx = p->nx, ny = p->ny;
    double smax = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IX(i, j);
            if (!wet[k]) continue;
            double c = sqrt(p->g * H[k]);
            double us = dmax(fabs(ux[k]), fabs(uy[k])) + c;
            double upx = fabs(ux[k] + sgn(ax[k]) * sqrt(p->dx * fabs(ax[k])));
            double upy = fabs(uy[k] + sgn(ay[k]) * sqrt(p->dx * fabs(ay[k])));
            double s = dmax(us, dmax(upx, upy));
            if (s > smax) smax = s;
            if (s != s) smax = s; /* NaN propagates */
        }
    return smax;
}

/* tau = min(dt_max, K h / S), dt_max when no cell is wet, dt_fixed when set;
 * never past t_end. */
static double time_step(const orc_params* p, double smax, double t)
{
    double tau;
    if (p->dt_fixed > 0.0) tau = p->dt_fixed;
    else if (smax > 0.0) tau = dmin(p->dt_max, p->cfl * p->dx / smax);
    else tau = p->dt_max;
    if (p->t_end > 0.0 && t + tau > p->t_end) tau = p->t_end - t;
    return tau;
}

static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* Two-rarefaction approximate Riemann solution (Toro 2001, Ch. 10) for the
 * shallow-water Riemann problem (hl, ul | hr, ur), sampled on the face
 * xi = x/t = 0.  A side with depth <= eps is dry and gives the dry-bed fan.
 * Writes (h, u) of the sampled state. */
void orc_riemann(double g, double eps, double hl, double ul, double hr, double ur, double* out)
{
    int dl = !(hl > eps), dr = !(hr > eps);
    double h = 0.0, u = 0.0;
    if (dl && dr) { out[0] = 0.0; out[1] = 0.0; return; }
    double cl = dl ? 0.0 : sqrt(g * hl);
    double cr = dr ? 0.0 : sqrt(g * hr);
    if (dr) {                                  /* left wet, right dry */
        if (ul - cl >= 0.0) { h = hl; u = ul; }
        else if (ul + 2.0 * cl > 0.0) { double c = (ul + 2.0 * cl) / 3.0; h = c * c / g; u = c; }
    } else if (dl) {                           /* left dry, right wet */
        if (ur + cr <= 0.0) { h = hr; u = ur; }
        else if (ur - 2.0 * cr < 0.0) { double c = (2.0 * cr - ur) / 3.0; h = c * c / g; u = -c; }
    } else if (2.0 * (cl + cr) <= ur - ul) {   /* both wet, a dry middle opens */
        if (ul - cl >= 0.0) { h = hl; u = ul; }
        else if (ul + 2.0 * cl > 0.0) { double c = (ul + 2.0 * cl) / 3.0; h = c * c / g; u = c; }
        else if (ur + cr <= 0.0) { h = hr; u = ur; }
        else if (ur - 2.0 * cr < 0.0) { double c = (2.0 * cr - ur) / 3.0; h = c * c / g; u = -c; }
    } else {
        double us = 0.5 * (ul + ur) + cl - cr;
        double cs = 0.5 * (cl + cr) + 0.25 * (ul - ur);
        if (us >= 0.0) {
            if (ul - cl >= 0.0) { h = hl; u = ul; }
            else if (us - cs >= 0.0) { double c = (ul + 2.0 * cl) / 3.0; h = c * c / g; u = c; }
            else { h = cs * cs / g; u = us; }
        } else {
            if (ur + cr <= 0.0) { h = hr; u = ur; }
            else if (us + cs <= 0.0) { double c = (2.0 * cr - ur) / 3.0; h = c * c / g; u = -c; }
            else { h = cs * cs / g; u = us; }
        }
    }
    out[0] = h; out[1] = u;
}

/* Sum of the source rates at time t for one source entry. */
static double source_rate(const orc_sources* s, int m, double t)
{
    const double* row = s->hydro_tab + 4 * (size_t)s->hydro[m];
    double q;
    if (row[0] == 0.0) {
        double z = (t - row[2]) / row[3];
        q = row[1] * exp(-0.5 * z * z);
    } else {
        q = row[1];
    }
    return s->weight[m] * q;
}

/* A correction c of a net flux sum f, bounded by beta |f| when beta > 0:
 * min(max(c, -beta |f|), beta |f|) (beta <= 0: c unchanged). */
static double bounded(double c, double f, double beta)
{
    if (!(beta > 0.0)) return c;
    double lim = beta * fabs(f);
    return dmin(dmax(c, -lim), lim);
}

/* One full time step from (H, Qx, Qy) at time t to (Hn, Qxn, Qyn).
 * corr (may be NULL): three [ny][nx] planes added to each cell's net
 * face-flux sums (Fh, Fv_x, Fv_y) before the final update, the additive
 * sub-grid corrections of a learned closure of a coarse grid level; with
 * corr_bound > 0 each correction is first bounded by corr_bound times the
 * magnitude of the flux sum it corrects.
 * Returns 0 on success, -1 on allocation failure, -5 when tau <= 0. */
int orc_step_corr(const orc_params* p, const double* b, const double* nm, const unsigned char* solid_in,
                  const orc_sources* src, double t, const double* H, const double* Qx, const double* Qy,
                  double* Hn, double* Qxn, double* Qyn, orc_info* info, orc_stages* st, const double* corr,
                  double corr_bound)
{
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * (size_t)ny;
    const double h = p->dx, g = p->g, eps = p->eps;
    int rc = 0;
    unsigned char* solid = (unsigned char*)calloc(N, 1);
    unsigned char* wet = (unsigned char*)calloc(N, 1);
    unsigned char* wt = (unsigned char*)calloc(N, 1);
    double* w = (double*)calloc(N * 24, sizeof(double));
    if (!solid || !wet || !wt || !w) { rc = -1; goto done; }
    if (solid_in) memcpy(solid, solid_in, N);
    double *ux = w, *uy = w + N, *ax = w + 2 * N, *ay = w + 3 * N, *phi = w + 4 * N;
    double *usx = w + 5 * N, *usy = w + 6 * N, *hs = w + 7 * N;
    double *ax2 = w + 8 * N, *ay2 = w + 9 * N, *phi2 = w + 10 * N;
    double *utx = w + 11 * N, *uty = w + 12 * N, *uhx = w + 13 * N, *uhy = w + 14 * N;
    double *ht = w + 15 * N, *qtx = w + 16 * N, *qty = w + 17 * N, *upx = w + 18 * N, *upy = w + 19 * N;
    double *eta = w + 20 * N, *sig = w + 21 * N;

    /* 1. primitives */
    for (size_t k = 0; k < N; ++k) {
        wet[k] = (!solid[k] && H[k] > eps);
        ux[k] = wet[k] ? Qx[k] / H[k] : 0.0;
        uy[k] = wet[k] ? Qy[k] / H[k] : 0.0;
    }
    /* 2. forces at t_n */
    forces(p, H, ux, uy, wet, solid, b, nm, ax, ay, phi);
    /* 3. time step */
    double smax = max_speed(p, H, ux, uy, ax, ay, wet);
    double tau = time_step(p, smax, t);
    if (!(tau > 0.0)) { rc = -5; goto done; }
    const double th = 0.5 * tau;
    /* 4. predictor: U* and the particle-area change D -> H* */
    for (size_t k = 0; k < N; ++k) {
        usx[k] = wet[k] ? (ux[k] + th * ax[k]) / (1.0 + th * phi[k]) : 0.0;
        usy[k] = wet[k] ? (uy[k] + th * ay[k]) / (1.0 + th * phi[k]) : 0.0;
    }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IX(i, j);
            if (!wet[k]) { hs[k] = H[k]; continue; }
            double uW = (i > 0) ? usx[k - 1] : 0.0, uE = (i < nx - 1) ? usx[k + 1] : 0.0;
            double vS = (j > 0) ? usy[k - nx] : 0.0, vN = (j < ny - 1) ? usy[k + nx] : 0.0;
            double fxm = 0.5 * (uW + usx[k]), fxp = 0.5 * (usx[k] + uE);
            double fym = 0.5 * (vS + usy[k]), fyp = 0.5 * (usy[k] + vN);
            double D = ((fxp - fxm) + (fyp - fym)) / h;
            hs[k] = H[k] / dmax(0.5, 1.0 + th * D);
        }
    /* 5. forces at t_{n+1/2}, corrector and sources */
    forces(p, hs, usx, usy, wet, solid, b, nm, ax2, ay2, phi2);
    double *vxc = w + 22 * N, *vyc = w + 23 * N;
    for (size_t k = 0; k < N; ++k) { sig[k] = 0.0; vxc[k] = 0.0; vyc[k] = 0.0; }
    if (src)
        for (int m = 0; m < src->n; ++m) {
            size_t k = IX(src->ix[m], src->iy[m]);
            sig[k] = source_rate(src, m, t + th);   /* sigma at t_n + tau/2 */
            vxc[k] = src->vx[m];
            vyc[k] = src->vy[m];
        }
    double src_sum = 0.0;
    for (size_t k = 0; k < N; ++k) {
        utx[k] = wet[k] ? (ux[k] + tau * ax2[k]) / (1.0 + tau * phi2[k]) : 0.0;
        uty[k] = wet[k] ? (uy[k] + tau * ay2[k]) / (1.0 + tau * phi2[k]) : 0.0;
        uhx[k] = 0.5 * (ux[k] + utx[k]);
        uhy[k] = 0.5 * (uy[k] + uty[k]);
        /* particle mass plus source.  Inflow brings water with velocity V;
         * a drain takes water with the cell's velocity U~, and never more
         * than the cell holds: a drain that empties the cell (H + tau sigma
         * <= 0) leaves it without momentum. */
        double ts = tau * sig[k];
        double hp = H[k] + ts;
        ht[k] = dmax(0.0, hp);
        if (sig[k] > 0.0 || hp > 0.0) {
            qtx[k] = H[k] * utx[k] + (sig[k] > 0.0 ? ts * vxc[k] : ts * utx[k]);
            qty[k] = H[k] * uty[k] + (sig[k] > 0.0 ? ts * vyc[k] : ts * uty[k]);
        } else {
            qtx[k] = 0.0;
            qty[k] = 0.0;
        }
        /* rain, evaporation and infiltration (Eq. 1 sigma) on every non-wall
         * cell.  Rain adds water at rest; the losses take water with U~, at
         * most the depth the point source left (max(0, hp)). */
        if (!solid[k] && (p->rain != 0.0 || p->evap != 0.0 || p->infil != 0.0)) {
            double loss = p->evap + p->infil;
            double taken = dmin(tau * loss, dmax(0.0, hp));
            ht[k] = dmax(0.0, hp + tau * (p->rain - loss));
            qtx[k] = qtx[k] - taken * utx[k];
            qty[k] = qty[k] - taken * uty[k];
        }
        src_sum += ht[k] - H[k];
        wt[k] = (!solid[k] && ht[k] > eps);
        upx[k] = wt[k] ? qtx[k] / ht[k] : 0.0;
        upy[k] = wt[k] ? qty[k] / ht[k] : 0.0;
        eta[k] = ht[k] + b[k];
    }
    /* 6. Eulerian face fluxes */
    double* fx = st && st->fx ? st->fx : NULL;
    double* fy = st && st->fy ? st->fy : NULL;
    double* fxl = (double*)calloc(3 * (size_t)ny * (size_t)(nx + 1), sizeof(double));
    double* fyl = (double*)calloc(3 * (size_t)(ny + 1) * (size_t)nx, sizeof(double));
    if (!fxl || !fyl) { free(fxl); free(fyl); rc = -1; goto done; }
    const size_t NFX = (size_t)ny * (size_t)(nx + 1), NFY = (size_t)(ny + 1) * (size_t)nx;
    const double* fld[5] = {eta, uhx, uhy, upx, upy};
    for (int dir = 0; dir < 2; ++dir) {
        /* dir 0: faces between (i,j) and (i+1,j); dir 1: (i,j) and (i,j+1) */
        int ni = dir == 0 ? nx - 1 : nx, nj = dir == 0 ? ny : ny - 1;
        for (int j = 0; j < nj; ++j)
            for (int i = 0; i < ni; ++i) {
                size_t kl = IX(i, j), kr = dir == 0 ? IX(i + 1, j) : IX(i, j + 1);
                double FH = 0.0, FQx = 0.0, FQy = 0.0;
                if (!solid[kl] && !solid[kr]) {
                    /* neighbours along the face normal: l2 = before kl, r2 = after kr */
                    int hasl2 = dir == 0 ? (i > 0) : (j > 0);
                    int hasr2 = dir == 0 ? (i + 2 < nx) : (j + 2 < ny);
                    size_t kl2 = hasl2 ? (dir == 0 ? kl - 1 : kl - (size_t)nx) : kl;
                    size_t kr2 = hasr2 ? (dir == 0 ? kr + 1 : kr + (size_t)nx) : kr;
                    int limL = hasl2 && wt[kl2] && wt[kl] && wt[kr];
                    int limR = hasr2 && wt[kl] && wt[kr] && wt[kr2];
                    double wl[5], wr[5];
                    for (int q = 0; q < 5; ++q) {
                        const double* v = fld[q];
                        double sl = limL ? minmod(v[kl] - v[kl2], v[kr] - v[kl]) : 0.0;
                        double sr = limR ? minmod(v[kr] - v[kl], v[kr2] - v[kr]) : 0.0;
                        wl[q] = v[kl] + 0.5 * sl;
                        wr[q] = v[kr] - 0.5 * sr;
                    }
                    double bs = dmax(b[kl], b[kr]);
                    double hl = dmax(0.0, wl[0] - bs), hr = dmax(0.0, wr[0] - bs);
                    double un_l = dir == 0 ? wl[1] : wl[2], un_r = dir == 0 ? wr[1] : wr[2];
                    double rs[2];
                    orc_riemann(g, eps, hl, un_l, hr, un_r, rs);
                    FH = rs[0] * rs[1];
                    FQx = FH * (FH >= 0.0 ? wl[3] : wr[3]);
                    FQy = FH * (FH >= 0.0 ? wl[4] : wr[4]);
                }
                if (dir == 0) {
                    size_t f = (size_t)j * (size_t)(nx + 1) + (size_t)(i + 1);
                    fxl[f] = FH; fxl[NFX + f] = FQx; fxl[2 * NFX + f] = FQy;
                } else {
                    size_t f = (size_t)(j + 1) * (size_t)nx + (size_t)i;
                    fyl[f] = FH; fyl[NFY + f] = FQx; fyl[2 * NFY + f] = FQy;
                }
            }
    }
    /* 7. final update: H^{n+1} = max(0, H~ + (tau/h) Fh), Q^{n+1} */
    const double dth = tau / h;
    double mass = 0.0, clip = 0.0;
    int64_t nwet = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IX(i, j);
            size_t fw = (size_t)j * (size_t)(nx + 1) + (size_t)i, fe = fw + 1;
            size_t fs = (size_t)j * (size_t)nx + (size_t)i, fn = fs + (size_t)nx;
            double fh = (fxl[fw] - fxl[fe]) + (fyl[fs] - fyl[fn]);
            double fqx = (fxl[NFX + fw] - fxl[NFX + fe]) + (fyl[NFY + fs] - fyl[NFY + fn]);
            double fqy = (fxl[2 * NFX + fw] - fxl[2 * NFX + fe]) + (fyl[2 * NFY + fs] - fyl[2 * NFY + fn]);
            if (corr) {
                fh = fh + bounded(corr[k], fh, corr_bound);
                fqx = fqx + bounded(corr[N + k], fqx, corr_bound);
                fqy = fqy + bounded(corr[2 * N + k], fqy, corr_bound);
            }
            double hn = ht[k] + dth * fh;
            if (hn < 0.0) { clip += -hn; hn = 0.0; }
            Hn[k] = hn;
            if (hn > eps) {
                Qxn[k] = qtx[k] + dth * fqx;
                Qyn[k] = qty[k] + dth * fqy;
            } else {
                Qxn[k] = 0.0; Qyn[k] = 0.0;
            }
            mass += hn;
            if (hn > eps && !solid[k]) nwet++;
        }
    if (info) {
        info->tau = tau; info->t_new = t + tau; info->smax = smax;
        info->mass = mass * h * h; info->clip_vol = clip * h * h; info->src_vol = src_sum * h * h;
        info->wet = nwet;
    }
    if (st) {
#define CP(dst, srcp) if (st->dst) memcpy(st->dst, srcp, N * sizeof(double))
        CP(ux, ux); CP(uy, uy); CP(ax, ax); CP(ay, ay); CP(phi, phi);
        CP(usx, usx); CP(usy, usy); CP(hs, hs); CP(ax2, ax2); CP(ay2, ay2); CP(phi2, phi2);
        CP(utx, utx); CP(uty, uty); CP(uhx, uhx); CP(uhy, uhy); CP(ht, ht); CP(qtx, qtx);
        CP(qty, qty); CP(upx, upx); CP(upy, upy);
#undef CP
        if (fx) memcpy(fx, fxl, 3 * NFX * sizeof(double));
        if (fy) memcpy(fy, fyl, 3 * NFY * sizeof(double));
    }
    free(fxl); free(fyl);
done:
    free(solid); free(wet); free(wt); free(w);
    return rc;
}

int orc_step(const orc_params* p, const double* b, const double* nm, const unsigned char* solid_in,
             const orc_sources* src, double t, const double* H, const double* Qx, const double* Qy,
             double* Hn, double* Qxn, double* Qyn, orc_info* info, orc_stages* st)
{
    return orc_step_corr(p, b, nm, solid_in, src, t, H, Qx, Qy, Hn, Qxn, Qyn, info, st, NULL, 0.0);
}

/* Largest signal speed of a state, as used for tau (for initial checks). */
double orc_state_speed(const orc_params* p, const double* b, const double* nm,
                       const unsigned char* solid_in, const double* H, const double* Qx,
                       const double* Qy)
{
    const size_t N = (size_t)p->nx * (size_t)p->ny;
    unsigned char* solid = (unsigned char*)calloc(N, 1);
    unsigned char* wet = (unsigned char*)calloc(N, 1);
    double* w = (double*)calloc(N * 5, sizeof(double));
    double s = -1.0;
    if (solid && wet && w) {
        if (solid_in) memcpy(solid, solid_in, N);
        double *ux = w, *uy = w + N, *ax = w + 2 * N, *ay = w + 3 * N, *phi = w + 4 * N;
        for (size_t k = 0; k < N; ++k) {
            wet[k] = (!solid[k] && H[k] > p->eps);
            ux[k] = wet[k] ? Qx[k] / H[k] : 0.0;
            uy[k] = wet[k] ? Qy[k] / H[k] : 0.0;
        }
        forces(p, H, ux, uy, wet, solid, b, nm, ax, ay, phi);
        s = max_speed(p, H, ux, uy, ax, ay, wet);
    }
    free(solid); free(wet); free(w);
    return s;
}
