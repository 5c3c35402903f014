// Host side of libswe: contexts, device memory, host copies, tensor maps,
// tiling, CUDA graphs and the C ABI declared in include/swe.h.
#include <algorithm>
#include <cmath>
#include <map>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/swe.h"
#include "swe_launch.h"
#include "swe_ptx.cuh"

using namespace swe;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(SWE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

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

bool finite_all(const double* a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

enum StageField {
    SF_UX, SF_UY, SF_AX, SF_AY, SF_PHI, SF_USX, SF_USY, SF_HS, SF_AX2, SF_AY2, SF_PHI2, SF_UTX, SF_UTY,
    SF_UHX, SF_UHY, SF_HT, SF_QTX, SF_QTY, SF_UPX, SF_UPY, SF_SIG, SF_SVX, SF_SVY,
    SF_FX0, SF_FX1, SF_FX2, SF_FY0, SF_FY1, SF_FY2, SF_COUNT
};

}  // namespace

void swe::set_last_error(const char* msg) { g_err = msg; }

struct swe_ctx {
    swe_params p;
    int dev = 0;
    int esz = 4;
    int pitch = 0, rows = 0;
    size_t plane = 0;
    void* f[8 + 2 * NACC] = {};  // H0 Qx0 Qy0 H1 Qx1 Qy1 b n, then (fused) ax0 ay0 ax1 ay1
    Ctl* ctl = nullptr;
    Ctl* ctl_host = nullptr;
    Part* parts = nullptr;
    Part* parts2 = nullptr;
    int parts_cap = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    // fused tiling
    int seg_h = 0, ntx = 0, nty = 0, nitems = 0;
    int sm_count = 0, occ = 0;
    // sources
    int nsrc = 0, nh = 0;
    int* d_scell = nullptr;
    int* d_shydro = nullptr;
    double* d_sw = nullptr;
    double* d_svx = nullptr;
    double* d_svy = nullptr;
    double* d_hydro = nullptr;
    SrcEntry* d_entries = nullptr;
    int* d_src_off = nullptr;
    // terrain copy (to reopen gates) and gate state
    std::vector<double> h_b;
    std::vector<uint8_t> h_solid;
    // staged intermediates
    void* scr[SF_COUNT] = {};
    // FP64 staging for host copies
    double* staging = nullptr;
    size_t staging_bytes = 0;
    int* d_tmp_i = nullptr;
    double* d_tmp_d = nullptr;
    size_t tmp_cap = 0;
    CUtensorMap tmH[2], tmQx[2], tmQy[2], tmB, tmN;
    CUtensorMap tmA[2][NACC];
    cudaGraphExec_t gexec = nullptr;
    int gsteps = 0;
    bool has_state = false;
    // host copies of the sources (to rebuild the per-item tables on retiling)
    std::vector<int32_t> hs_ix, hs_iy, hs_hy;
    std::vector<double> hs_w, hs_vx, hs_vy;
    unsigned long long generation = 0;  // bumps when device pointers or tiling change
    // learned closure (attached network, its normalisation, buffers)
    swe_cnn* cnn = nullptr;
    float* d_norm = nullptr;   // 16 floats: in mu[5], in sd[5], out mu[3], out sd[3]
    void* d_feat = nullptr;    // BF16 [ny][nx][16]
    void* d_corr = nullptr;    // 3 padded planes
    double* d_acc = nullptr;
    double corr_bound = 0.0;   // > 0: corrections bounded by this fraction of the plain flux sums
    cudaGraphExec_t cexec = nullptr;
    int csteps = 0;
    // wet-block stamps (skip_dry)
    long long* d_act = nullptr;
    int act_nbx = 0, act_nby = 0;
    unsigned char* d_hist = nullptr;  // per-item skip history (parts_cap bytes)
};

namespace {

template <class T>
Grid<T> grid_of(const swe_ctx* c) {
    Grid<T> g;
    g.nx = c->p.nx;
    g.ny = c->p.ny;
    g.pitch = c->pitch;
    for (int b = 0; b < 2; ++b) {
        g.H[b] = (T*)c->f[3 * b + 0];
        g.Qx[b] = (T*)c->f[3 * b + 1];
        g.Qy[b] = (T*)c->f[3 * b + 2];
    }
    g.b = (T*)c->f[6];
    g.n = (T*)c->f[7];
    for (int b = 0; b < 2; ++b)
        for (int q = 0; q < NACC; ++q) g.A[b][q] = (T*)c->f[8 + NACC * b + q];
    return g;
}

template <class T>
Phys<T> phys_of(const swe_params& p) {
    Phys<T> P;
    P.g = (T)p.g;
    P.h = (T)p.dx;
    P.eps = (T)p.eps_dry;
    P.nu = (T)p.nu;
    P.f = (T)p.coriolis_f;
    P.wx = (T)p.wind_x;
    P.wy = (T)p.wind_y;
    P.ca = (T)p.c_a;
    P.ra = (T)p.rho_air_over_rho;
    P.rain = (T)p.rain_rate;
    P.loss = (T)(p.evap_rate + p.infil_rate);
    P.dist = (p.rain_rate != 0.0 || p.evap_rate != 0.0 || p.infil_rate != 0.0) ? 1 : 0;
    phys_derive(P);
    return P;
}

StepP stepp_of(const swe_params& p) {
    StepP s;
    s.dx = p.dx;
    s.cfl = p.cfl;
    s.dt_max = p.dt_max;
    s.dt_fixed = p.dt_fixed;
    return s;
}

template <class T>
StagedArgs<T> staged_args(const swe_ctx* c) {
    StagedArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.g = grid_of<T>(c);
    a.P = phys_of<T>(c->p);
    a.sp = stepp_of(c->p);
    a.ctl = c->ctl;
    a.parts = c->parts;
    a.parts2 = c->parts2;
    T** fields[] = {&a.ux, &a.uy, &a.ax, &a.ay, &a.phi, &a.usx, &a.usy, &a.hs, &a.ax2, &a.ay2, &a.phi2,
                    &a.utx, &a.uty, &a.uhx, &a.uhy, &a.ht, &a.qtx, &a.qty, &a.upx, &a.upy, &a.sig,
                    &a.svx, &a.svy, &a.fx[0], &a.fx[1], &a.fx[2], &a.fy[0], &a.fy[1], &a.fy[2]};
    for (int k = 0; k < SF_COUNT; ++k) *fields[k] = (T*)c->scr[k];
    a.s_cell = c->d_scell;
    a.s_hydro = c->d_shydro;
    a.s_w = c->d_sw;
    a.s_vx = c->d_svx;
    a.s_vy = c->d_svy;
    a.nsrc = c->nsrc;
    a.hydro = c->d_hydro;
    a.nh = c->nh;
    a.act = c->d_act;
    a.act_nbx = c->act_nbx;
    a.hist = c->d_hist;
    a.nhist = c->d_hist ? c->parts_cap : 0;
    a.open_ring = c->p.ghost_ring == 2 ? 1 : 0;
    return a;
}

template <class T>
FusedArgs<T> fused_args(const swe_ctx* c, bool closed = false) {
    FusedArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    for (int b = 0; b < 2; ++b) {
        a.tmH[b] = c->tmH[b];
        a.tmQx[b] = c->tmQx[b];
        a.tmQy[b] = c->tmQy[b];
    }
    a.tmB = c->tmB;
    a.tmN = c->tmN;
    for (int b = 0; b < 2; ++b)
        for (int q = 0; q < NACC; ++q) a.tmA[b][q] = c->tmA[b][q];
    a.g = grid_of<T>(c);
    a.P = phys_of<T>(c->p);
    a.sp = stepp_of(c->p);
    a.ctl = c->ctl;
    a.parts = c->parts;
    a.src = c->d_entries;
    a.src_off = c->d_src_off;
    a.hydro = c->d_hydro;
    a.nh = c->nh;
    a.ntx = c->ntx;
    a.seg_h = c->seg_h;
    a.nitems = c->nitems;
    a.corr = closed ? (const T*)c->d_corr : nullptr;
    a.corr_bound = (T)c->corr_bound;
    a.act = c->d_act;
    a.act_nbx = c->act_nbx;
    // closed steps stamp but never skip; rain wets dry tiles and the losses
    // change thin films, so distributed sources switch skipping off
    a.skip = (c->d_act && !closed && !a.P.dist) ? 1 : 0;
    a.hist = c->d_hist;
    a.corr_plane = (size_t)c->pitch * (size_t)c->rows;
    a.open_ring = c->p.ghost_ring == 2 ? 1 : 0;
    return a;
}

bool is64(const swe_ctx* c) { return c->p.precision == SWE_F64; }

// Launch-cost model of the fused kernel: waves of CTAs times rows per CTA.
// With dry-tile skipping the few wet items set the step time (each streams
// its rows one after another), so segments stay at most 256 rows high.
void choose_tiling(swe_ctx* c) {
    const int nx = c->p.nx, ny = c->p.ny;
    c->ntx = (nx + TW - 1) / TW;
    int best = 0;
    double best_cost = 1e300;
    // candidates: 8, 12, 16, 24, then every multiple of 16 up to 1024 (fine
    // enough to fill the last wave: a 4096-row grid gets 352-row segments,
    // 0.95 waves, instead of 384-row ones, 0.87)
    std::vector<int> cand = {8, 12, 16, 24};
    for (int sh = 32; sh <= 1024; sh += 16) cand.push_back(sh);
    const int slots = std::max(1, c->sm_count * std::max(1, c->occ));
    const int cap = c->p.skip_dry ? 256 : 1 << 30;
    for (int sh : cand) {
        if ((sh > ny || sh > cap) && best != 0) break;
        const long long items = (long long)c->ntx * ((ny + sh - 1) / sh);
        const double waves = std::ceil((double)items / slots);
        const double cost = waves * (std::min(sh, ny) + 2 * HALO);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = sh;
        }
    }
    c->seg_h = c->p.seg_h > 0 ? c->p.seg_h : best;
    c->nty = (ny + c->seg_h - 1) / c->seg_h;
    c->nitems = c->ntx * c->nty;
}

int encode_map(swe_ctx* c, CUtensorMap* m, void* base) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(SWE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {(cuuint64_t)(c->p.nx + 2 * PAD), (cuuint64_t)(c->p.ny + 2 * PAD)};
    cuuint64_t strides[1] = {(cuuint64_t)c->pitch * (cuuint64_t)c->esz};
    cuuint32_t box[2] = {(cuuint32_t)WIN, (cuuint32_t)RB};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, is64(c) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SWE_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return SWE_OK;
}

int ensure_staging(swe_ctx* c, size_t bytes) {
    if (c->staging_bytes >= bytes) return SWE_OK;
    if (c->staging) {
        CK(cudaStreamSynchronize(c->st));
        cudaFree(c->staging);
        c->staging = nullptr;
        c->staging_bytes = 0;
    }
    if (cudaMalloc(&c->staging, bytes) != cudaSuccess) return fail(SWE_ERR_OOM, "staging allocation failed");
    c->staging_bytes = bytes;
    return SWE_OK;
}

int ensure_tmp(swe_ctx* c, size_t n) {
    if (c->tmp_cap >= n) return SWE_OK;
    CK(cudaStreamSynchronize(c->st));
    cudaFree(c->d_tmp_i);
    cudaFree(c->d_tmp_d);
    c->d_tmp_i = nullptr;
    c->d_tmp_d = nullptr;
    c->tmp_cap = 0;
    if (cudaMalloc(&c->d_tmp_i, n * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_tmp_d, n * sizeof(double)) != cudaSuccess)
        return fail(SWE_ERR_OOM, "temporary allocation failed");
    c->tmp_cap = n;
    return SWE_OK;
}

// Host FP64 [ny][nx] -> padded device field (through the FP64 staging);
// with flag, non-finite (and, with check_neg, negative) values are flagged.
int upload_field(swe_ctx* c, const double* host, void* dev, unsigned* flag = nullptr, int check_neg = 0) {
    const size_t n = (size_t)c->p.nx * c->p.ny;
    int rc = ensure_staging(c, n * sizeof(double));
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->staging, host, n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(is64(c) ? launch_pack<double>(c->staging, (double*)dev, c->p.nx, c->p.ny, c->pitch, c->st, flag, check_neg)
               : launch_pack<float>(c->staging, (float*)dev, c->p.nx, c->p.ny, c->pitch, c->st, flag, check_neg));
    return SWE_OK;
}

// Host [ny][nx] in the context's precision -> padded device field by one
// 2-D copy (no staging, no conversion); the values are checked by the speed
// pass that follows (launch_state_speed with check).
int upload_native(swe_ctx* c, const void* host, void* dev) {
    const size_t row = (size_t)c->p.nx * c->esz;
    char* dst = (char*)dev + ((size_t)PAD * c->pitch + PAD) * c->esz;
    CK(cudaMemcpy2DAsync(dst, (size_t)c->pitch * c->esz, host, row, row, (size_t)c->p.ny, cudaMemcpyHostToDevice,
                         c->st));
    return SWE_OK;
}

// Padded device field (base of the interior shifted by (ox, oy)) -> host
// FP64 [ny][nx], both sizes given.
int download_field(swe_ctx* c, const void* dev, double* host, int nx, int ny, long long shift_elems) {
    const size_t n = (size_t)nx * ny;
    int rc = ensure_staging(c, n * sizeof(double));
    if (rc) return rc;
    if (is64(c))
        CK(launch_unpack<double>((const double*)dev + shift_elems, c->staging, nx, ny, c->pitch, c->st));
    else
        CK(launch_unpack<float>((const float*)dev + shift_elems, c->staging, nx, ny, c->pitch, c->st));
    CK(cudaMemcpyAsync(host, c->staging, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    return SWE_OK;
}

int read_ctl(swe_ctx* c) {
    CK(cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SWE_OK;
}

int state_speed(swe_ctx* c, int check = 0) {
    if (is64(c)) CK(launch_state_speed<double>(staged_args<double>(c), c->st, check));
    else CK(launch_state_speed<float>(staged_args<float>(c), c->st, check));
    return SWE_OK;
}

void drop_graph(swe_ctx* c) {
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        c->gsteps = 0;
    }
}

int launch_one_step(swe_ctx* c) {
    if (c->p.mode == SWE_STAGED) {
        if (is64(c)) CK(launch_staged<double>(staged_args<double>(c), c->st));
        else CK(launch_staged<float>(staged_args<float>(c), c->st));
    } else {
        if (c->p.ghost_ring == 2) {  // open boundary: extend the state into the ring
            if (is64(c)) {
                CK(launch_ring_outflow<double>(grid_of<double>(c), c->ctl, c->st));
                CK(launch_band_acc<double>(staged_args<double>(c), c->st));
            } else {
                CK(launch_ring_outflow<float>(grid_of<float>(c), c->ctl, c->st));
                CK(launch_band_acc<float>(staged_args<float>(c), c->st));
            }
        }
        if (is64(c)) CK(launch_fused<double>(fused_args<double>(c), c->st));
        else CK(launch_fused<float>(fused_args<float>(c), c->st));
    }
    return SWE_OK;
}

// Per-work-item source lists of the fused kernel, in window coordinates and
// sorted by (row, column).
int build_source_tables(swe_ctx* c, const int32_t* ix, const int32_t* iy, const double* w, const double* vx,
                        const double* vy, const int32_t* hy) {
    std::vector<std::vector<SrcEntry>> per(c->nitems);
    for (int m = 0; m < c->nsrc; ++m) {
        const int sx_lo = std::max(0, (ix[m] + HALO - (WIN - 1) + TW - 1) / TW - 1);
        const int sx_hi = std::min(c->ntx - 1, (ix[m] + HALO) / TW);
        const int gy_lo = std::max(0, (iy[m] - c->seg_h - HALO) / c->seg_h - 1);
        const int gy_hi = std::min(c->nty - 1, (iy[m] + HALO) / c->seg_h);
        for (int sy = gy_lo; sy <= gy_hi; ++sy)
            for (int sx = sx_lo; sx <= sx_hi; ++sx) {
                const int x0 = sx * TW, y0 = sy * c->seg_h;
                const int sh = std::min(c->seg_h, c->p.ny - y0);
                const int r = iy[m] - y0 + HALO, col = ix[m] - x0 + HALO;
                if (r < 0 || r >= sh + 2 * HALO || col < 0 || col >= WIN) continue;
                SrcEntry e;
                e.r = (short)r;
                e.c = (short)col;
                e.hydro = hy[m];
                e.w = w[m];
                e.vx = vx ? vx[m] : 0.0;
                e.vy = vy ? vy[m] : 0.0;
                per[sy * c->ntx + sx].push_back(e);
            }
    }
    std::vector<int> off(c->nitems + 1, 0);
    std::vector<SrcEntry> all;
    for (int i = 0; i < c->nitems; ++i) {
        std::sort(per[i].begin(), per[i].end(), [](const SrcEntry& a, const SrcEntry& b) {
            return a.r != b.r ? a.r < b.r : a.c < b.c;
        });
        off[i] = (int)all.size();
        all.insert(all.end(), per[i].begin(), per[i].end());
    }
    off[c->nitems] = (int)all.size();
    cudaFree(c->d_entries);
    cudaFree(c->d_src_off);
    c->d_entries = nullptr;
    c->d_src_off = nullptr;
    if (cudaMalloc(&c->d_src_off, off.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_entries, std::max<size_t>(1, all.size()) * sizeof(SrcEntry)) != cudaSuccess)
        return fail(SWE_ERR_OOM, "source table allocation failed");
    CK(cudaMemcpy(c->d_src_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!all.empty())
        CK(cudaMemcpy(c->d_entries, all.data(), all.size() * sizeof(SrcEntry), cudaMemcpyHostToDevice));
    return SWE_OK;
}

// Bed values of the given cells (walls where closed) -> device.
int apply_beds(swe_ctx* c, const std::vector<int>& cells) {
    if (cells.empty()) return SWE_OK;
    int rc = ensure_tmp(c, cells.size());
    if (rc) return rc;
    std::vector<int> idx(cells.size());
    std::vector<double> val(cells.size());
    for (size_t m = 0; m < cells.size(); ++m) {
        const int i = cells[m] % c->p.nx, j = cells[m] / c->p.nx;
        idx[m] = (j + PAD) * c->pitch + (i + PAD);
        val[m] = c->h_solid[cells[m]] ? WALL_BED : c->h_b[cells[m]];
    }
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpy(c->d_tmp_i, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_tmp_d, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (is64(c)) CK(launch_scatter<double>((double*)c->f[6], c->d_tmp_i, c->d_tmp_d, (int)idx.size(), c->st));
    else CK(launch_scatter<float>((float*)c->f[6], c->d_tmp_i, c->d_tmp_d, (int)idx.size(), c->st));
    return SWE_OK;
}

// Re-tile a fused context: new segment height, per-item source tables and
// partial-sum capacity.
int retile(swe_ctx* c, int seg_h) {
    c->p.seg_h = seg_h;
    choose_tiling(c);
    if (c->nitems > c->parts_cap) {
        CK(cudaStreamSynchronize(c->st));
        cudaFree(c->parts);
        cudaFree(c->parts2);
        c->parts = nullptr;
        c->parts2 = nullptr;
        c->parts_cap = c->nitems;
        if (cudaMalloc(&c->parts, c->parts_cap * sizeof(Part)) != cudaSuccess ||
            cudaMalloc(&c->parts2, c->parts_cap * sizeof(Part)) != cudaSuccess)
            return fail(SWE_ERR_OOM, "partials");
        if (c->d_act) {
            cudaFree(c->d_hist);
            c->d_hist = nullptr;
            if (cudaMalloc(&c->d_hist, c->parts_cap) != cudaSuccess) return fail(SWE_ERR_OOM, "skip history");
        }
    }
    // the items changed: no item has a skip history
    if (c->d_hist) CK(cudaMemsetAsync(c->d_hist, 0, c->parts_cap, c->st));
    drop_graph(c);
    c->generation++;
    const int n = c->nsrc;
    return build_source_tables(c, n ? c->hs_ix.data() : nullptr, n ? c->hs_iy.data() : nullptr,
                               n ? c->hs_w.data() : nullptr, n ? c->hs_vx.data() : nullptr,
                               n ? c->hs_vy.data() : nullptr, n ? c->hs_hy.data() : nullptr);
}

// Device copy of a context's current state (with its stored accelerations)
// and control block, for trial runs that must leave the state as it was.
struct Snapshot {
    void* planes[3 + NACC] = {};
    Ctl ctl;
    int buf = 0;
};

int snapshot_take(swe_ctx* c, Snapshot& sn) {
    int rc = read_ctl(c);
    if (rc) return rc;
    sn.ctl = *c->ctl_host;
    sn.buf = (int)(sn.ctl.step & 1);
    for (int k = 0; k < 3 + NACC; ++k) {
        void* src = k < 3 ? c->f[3 * sn.buf + k] : c->f[8 + NACC * sn.buf + (k - 3)];
        if (!src) continue;
        if (cudaMalloc(&sn.planes[k], c->plane) != cudaSuccess) return fail(SWE_ERR_OOM, "snapshot");
        CK(cudaMemcpyAsync(sn.planes[k], src, c->plane, cudaMemcpyDeviceToDevice, c->st));
    }
    return SWE_OK;
}

int snapshot_restore(swe_ctx* c, Snapshot& sn) {
    for (int k = 0; k < 3 + NACC; ++k) {
        void* dst = k < 3 ? c->f[3 * sn.buf + k] : c->f[8 + NACC * sn.buf + (k - 3)];
        if (dst && sn.planes[k])
            CK(cudaMemcpyAsync(dst, sn.planes[k], c->plane, cudaMemcpyDeviceToDevice, c->st));
    }
    *c->ctl_host = sn.ctl;
    CK(cudaMemcpyAsync(c->ctl, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st));
    // the other buffer holds trial steps: no item may rely on it
    if (c->d_hist) CK(cudaMemsetAsync(c->d_hist, 0, c->parts_cap, c->st));
    CK(cudaStreamSynchronize(c->st));
    return SWE_OK;
}

void snapshot_free(Snapshot& sn) {
    for (void*& q : sn.planes) {
        cudaFree(q);
        q = nullptr;
    }
}

const int kTileCandidates[] = {16, 32, 64, 128, 192, 256, 384, 512, 768, 1024};

}  // namespace

struct swe_batch {
    std::vector<swe_ctx*> ctx;
    bool f64 = false;
    int dev = 0;
    cudaStream_t st = nullptr;
    void* d_descs = nullptr;
    int2* d_work = nullptr;
    int nwork = 0;
    BatchCtl* bc = nullptr;
    int grid = 0;
    std::vector<unsigned long long> gen;
    struct Ev {
        long long step;
        int scen;
        int cell;
        uint8_t closed;
    };
    std::vector<Ev> events;   // sorted by step
    int* d_ev_idx = nullptr;  // padded bed index of each event
    double* d_ev_val = nullptr;
    long long step = 0;       // batch steps taken since creation
    cudaGraphExec_t gexec = nullptr;  // graph of a step window with gate events
    long long gbase = -1;
    int gsteps = 0;
    std::map<int, cudaGraphExec_t> plain;  // event-free windows, by length
};

namespace {

void batch_drop_graph(swe_batch* b) {
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        b->gsteps = 0;
        b->gbase = -1;
    }
    for (auto& kv : b->plain) cudaGraphExecDestroy(kv.second);
    b->plain.clear();
}

// Scenario descriptors and the work list (largest items first, so the
// persistent CTAs end together).
int batch_build(swe_batch* b) {
    const int n = (int)b->ctx.size();
    const size_t dsz = b->f64 ? sizeof(FusedArgs<double>) : sizeof(FusedArgs<float>);
    std::vector<unsigned char> host(dsz * n);
    struct W {
        long long cost;
        int s, i;
    };
    std::vector<W> work;
    for (int k = 0; k < n; ++k) {
        swe_ctx* c = b->ctx[k];
        if (b->f64) {
            FusedArgs<double> a = fused_args<double>(c);
            std::memcpy(host.data() + dsz * k, &a, dsz);
        } else {
            FusedArgs<float> a = fused_args<float>(c);
            std::memcpy(host.data() + dsz * k, &a, dsz);
        }
        for (int i = 0; i < c->nitems; ++i) {
            const int x0 = (i % c->ntx) * TW, y0 = (i / c->ntx) * c->seg_h;
            const long long cost = (long long)(std::min(TW, c->p.nx - x0) + 2 * HALO) *
                                   (std::min(c->seg_h, c->p.ny - y0) + 2 * HALO + 5);
            work.push_back({cost, k, i});
        }
    }
    std::stable_sort(work.begin(), work.end(), [](const W& x, const W& y) { return x.cost > y.cost; });
    std::vector<int2> wl(work.size());
    for (size_t m = 0; m < work.size(); ++m) wl[m] = make_int2(work[m].s, work[m].i);
    CK(cudaStreamSynchronize(b->st));
    cudaFree(b->d_descs);
    cudaFree(b->d_work);
    b->d_descs = nullptr;
    b->d_work = nullptr;
    if (cudaMalloc(&b->d_descs, host.size()) != cudaSuccess ||
        cudaMalloc((void**)&b->d_work, wl.size() * sizeof(int2)) != cudaSuccess)
        return fail(SWE_ERR_OOM, "batch descriptors");
    CK(cudaMemcpy(b->d_descs, host.data(), host.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_work, wl.data(), wl.size() * sizeof(int2), cudaMemcpyHostToDevice));
    b->nwork = (int)wl.size();
    b->gen.resize(n);
    for (int k = 0; k < n; ++k) b->gen[k] = b->ctx[k]->generation;
    batch_drop_graph(b);
    return SWE_OK;
}

int batch_launch_step(swe_batch* b) {
    if (b->f64) {
        BatchArgs<double> a{(const FusedArgs<double>*)b->d_descs, b->d_work, b->nwork, b->bc};
        CK(launch_fused_batch<double>(a, b->grid, b->st));
    } else {
        BatchArgs<float> a{(const FusedArgs<float>*)b->d_descs, b->d_work, b->nwork, b->bc};
        CK(launch_fused_batch<float>(a, b->grid, b->st));
    }
    return SWE_OK;
}

// Gate events scheduled before batch step `s`: new beds, then the signal
// speed of each touched scenario (as swe_set_solid does for one context).
int batch_launch_events(swe_batch* b, long long s) {
    auto lo = std::lower_bound(b->events.begin(), b->events.end(), s,
                               [](const swe_batch::Ev& e, long long v) { return e.step < v; });
    auto hi = std::upper_bound(b->events.begin(), b->events.end(), s,
                               [](long long v, const swe_batch::Ev& e) { return v < e.step; });
    if (lo == hi) return SWE_OK;
    std::vector<int> scen;
    for (auto it = lo; it != hi; ++it) {
        const size_t m = (size_t)(it - b->events.begin());
        swe_ctx* c = b->ctx[it->scen];
        if (b->f64) CK(launch_scatter<double>((double*)c->f[6], b->d_ev_idx + m, b->d_ev_val + m, 1, b->st));
        else CK(launch_scatter<float>((float*)c->f[6], b->d_ev_idx + m, b->d_ev_val + m, 1, b->st));
        if (std::find(scen.begin(), scen.end(), it->scen) == scen.end()) scen.push_back(it->scen);
    }
    for (int k : scen) {
        swe_ctx* c = b->ctx[k];
        if (b->f64) CK(launch_state_speed<double>(staged_args<double>(c), b->st));
        else CK(launch_state_speed<float>(staged_args<float>(c), b->st));
    }
    return SWE_OK;
}

// One closed coarse step: features of the current state, network, mass-
// centred corrections, fused step with the corrections in its final update.
int launch_closed_step(swe_ctx* c) {
    const float* nin = c->d_norm;
    const float* nout = c->d_norm + 10;
    if (is64(c)) {
        CK(launch_features<double>(grid_of<double>(c), c->ctl, (double)c->p.eps_dry, nin, c->d_feat, c->st));
    } else {
        CK(launch_features<float>(grid_of<float>(c), c->ctl, (float)c->p.eps_dry, nin, c->d_feat, c->st));
    }
    int rc = cnn_forward_on(c->cnn, c->d_feat, c->st);
    if (rc) return rc;
    const size_t plane = (size_t)c->pitch * (size_t)c->rows;
    if (is64(c)) {
        CK(launch_corrections<double>(grid_of<double>(c), c->ctl, (double)c->p.eps_dry, cnn_output(c->cnn), nout,
                                      (double*)c->d_corr, plane, c->d_acc, c->st));
        CK(launch_fused<double>(fused_args<double>(c, true), c->st));
    } else {
        CK(launch_corrections<float>(grid_of<float>(c), c->ctl, (float)c->p.eps_dry, cnn_output(c->cnn), nout,
                                     (float*)c->d_corr, plane, c->d_acc, c->st));
        CK(launch_fused<float>(fused_args<float>(c, true), c->st));
    }
    return SWE_OK;
}

int batch_sync_all(swe_batch* b) {
    for (swe_ctx* c : b->ctx) CK(cudaStreamSynchronize(c->st));
    CK(cudaStreamSynchronize(b->st));
    return SWE_OK;
}

}  // namespace

// Reset the control block to time t, upload the three fields with
// upload(k, check_neg) (k = 0: H, 1: Qx, 2: Qy), check them on the device
// and compute the first time step's signal speed.  With speed_checks the
// uploads leave the checks to the speed pass, which then runs first.
template <class Up>
int set_state_with(swe_ctx* c, double t, Up upload, bool speed_checks = false) {
    if (!std::isfinite(t)) return fail(SWE_ERR_NONFINITE, "t not finite");
    CK(cudaSetDevice(c->dev));
    // the values are checked on the device while they are copied in
    Ctl h;
    std::memset(&h, 0, sizeof(h));
    h.t = t;
    *c->ctl_host = h;
    CK(cudaMemcpyAsync(c->ctl, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st));
    int rc = upload(0, 1);
    if (!rc) rc = upload(1, 0);
    if (!rc) rc = upload(2, 0);
    if (rc) return rc;
    if (speed_checks) {
        rc = state_speed(c, 1);
        if (rc) return rc;
    }
    rc = read_ctl(c);
    if (rc) return rc;
    if (c->ctl_host->err) {
        const unsigned e = c->ctl_host->err;
        c->has_state = false;
        if (e & 1u) return fail(SWE_ERR_NONFINITE, "state not finite (in FP64 or after conversion)");
        return fail(SWE_ERR_ARG, "negative depth");
    }
    if (!speed_checks) {
        rc = state_speed(c);
        if (rc) return rc;
    }
    c->has_state = true;
    return SWE_OK;
}

// A bounded wait on an mbarrier phase that nothing completes: the wait the
// step kernels use for their TMA rows, run out on purpose so the error path
// (error bit, status to the host, usable context) can be checked without a
// fault or a hang.
static __global__ void k_wait_probe(unsigned* err, unsigned long long limit_ns) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        swe::mbar_init(&bar, 1);
        swe::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !swe::mbar_wait_bounded(&bar, 0u, limit_ns)) atomicOr(err, (unsigned)swe::ERR_TIMEOUT);
    __syncthreads();
}

extern "C" {

void swe_params_default(swe_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->precision = SWE_F32;
    p->mode = SWE_FUSED;
    p->g = 9.81;
    p->cfl = 0.3;
    p->eps_dry = 1e-4;
    p->dt_max = 1.0;
    p->rho_air_over_rho = 1.225e-3;
}

const char* swe_status_str(int s) {
    switch (s) {
        case SWE_OK: return "ok";
        case SWE_ERR_ARG: return "invalid argument";
        case SWE_ERR_CUDA: return "CUDA error";
        case SWE_ERR_OOM: return "out of memory";
        case SWE_ERR_NONFINITE: return "non-finite value";
        case SWE_ERR_DT: return "time step not positive";
        case SWE_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        case SWE_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

const char* swe_last_error(void) { return g_err.c_str(); }

int swe_create(const swe_params* p, swe_ctx** out) {
    if (!p || !out) return fail(SWE_ERR_ARG, "null argument");
    *out = nullptr;
    if (p->nx < 1 || p->ny < 1 || p->nx > (1 << 20) || p->ny > (1 << 20) ||
        (double)p->nx * p->ny > 4.0e9)
        return fail(SWE_ERR_ARG, "grid size out of range");
    if (!(p->dx > 0.0) || !(p->g > 0.0) || !(p->cfl > 0.0 && p->cfl <= 1.0) || !(p->eps_dry >= 0.0) ||
        !(p->dt_max > 0.0) || !(p->dt_fixed >= 0.0) || !(p->nu >= 0.0) || !(p->c_a >= 0.0) ||
        !(p->rho_air_over_rho >= 0.0) || !std::isfinite(p->coriolis_f) || !std::isfinite(p->wind_x) ||
        !std::isfinite(p->wind_y))
        return fail(SWE_ERR_ARG, "physical or numerical parameter out of range");
    if (p->precision != SWE_F32 && p->precision != SWE_F64) return fail(SWE_ERR_ARG, "precision");
    if (p->mode != SWE_FUSED && p->mode != SWE_STAGED) return fail(SWE_ERR_ARG, "mode");
    if (p->seg_h < 0 || p->seg_h > 32768 || p->tile_w < 0) return fail(SWE_ERR_ARG, "tiling");
    if (p->tile_w != 0 && p->tile_w != TW) return fail(SWE_ERR_ARG, "tile_w must be 0 or 116");
    if (p->skip_dry != 0 && p->skip_dry != 1) return fail(SWE_ERR_ARG, "skip_dry must be 0 or 1");
    if (p->skip_dry && p->mode != SWE_FUSED) return fail(SWE_ERR_ARG, "skip_dry needs SWE_FUSED");
    if (p->ghost_ring < 0 || p->ghost_ring > 2) return fail(SWE_ERR_ARG, "ghost_ring must be 0, 1 or 2");
    if (!(p->rain_rate >= 0.0 && p->rain_rate < 1.0) || !(p->evap_rate >= 0.0 && p->evap_rate < 1.0) ||
        !(p->infil_rate >= 0.0 && p->infil_rate < 1.0))
        return fail(SWE_ERR_ARG, "rain, evaporation and infiltration rates must lie in [0, 1) m/s");
    if (p->ghost_ring && p->mode != SWE_FUSED) return fail(SWE_ERR_ARG, "ghost_ring needs SWE_FUSED");
    if (p->ghost_ring && p->skip_dry)
        return fail(SWE_ERR_ARG, "skip_dry needs wall boundaries (ghost cells are not stamped)");
    swe_ctx* c = new (std::nothrow) swe_ctx();
    if (!c) return fail(SWE_ERR_OOM, "context");
    c->p = *p;
    c->esz = p->precision == SWE_F64 ? 8 : 4;
    c->pitch = ((p->nx + 2 * PAD + 31) / 32) * 32;
    c->rows = p->ny + 2 * PAD;
    c->plane = (size_t)c->pitch * c->rows * c->esz;
    auto bail = [&](int code, const std::string& m) {
        swe_destroy(c);
        return fail(code, m);
    };
    if (cudaGetDevice(&c->dev) != cudaSuccess) return bail(SWE_ERR_CUDA, "no CUDA device");
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->dev) != cudaSuccess) return bail(SWE_ERR_CUDA, "device properties");
    c->sm_count = prop.multiProcessorCount;
    if (p->cuda_stream) {
        c->st = (cudaStream_t)p->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess)
            return bail(SWE_ERR_CUDA, "stream creation");
        c->own_stream = true;
    }
    // stored accelerations: every fused context (with a ghost ring, the band
    // a fill changes is refreshed after each fill, launch_band_acc)
    const int nplanes = p->mode == SWE_FUSED ? 8 + 2 * NACC : 8;
    for (int k = 0; k < nplanes; ++k) {
        if (cudaMalloc(&c->f[k], c->plane) != cudaSuccess) return bail(SWE_ERR_OOM, "state allocation");
        if (cudaMemsetAsync(c->f[k], 0, c->plane, c->st) != cudaSuccess) return bail(SWE_ERR_CUDA, "memset");
    }
    cudaError_t e = is64(c) ? launch_fill_bed<double>((double*)c->f[6], p->nx, p->ny, c->pitch, c->st)
                            : launch_fill_bed<float>((float*)c->f[6], p->nx, p->ny, c->pitch, c->st);
    if (e != cudaSuccess) return bail(SWE_ERR_CUDA, "fill bed");
    if (cudaMalloc(&c->ctl, sizeof(Ctl)) != cudaSuccess) return bail(SWE_ERR_OOM, "control block");
    if (cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), c->st) != cudaSuccess) return bail(SWE_ERR_CUDA, "memset");
    if (cudaMallocHost(&c->ctl_host, sizeof(Ctl)) != cudaSuccess) return bail(SWE_ERR_OOM, "pinned control block");
    // occupancy of the fused kernel decides the tiling
    c->occ = 1;
    if (p->mode == SWE_FUSED) {
        e = is64(c) ? prepare_fused<double>(&c->occ) : prepare_fused<float>(&c->occ);
        if (e != cudaSuccess) return bail(SWE_ERR_CUDA, std::string("fused kernel setup: ") + cudaGetErrorString(e));
        if (c->occ < 1) return bail(SWE_ERR_CUDA, "fused kernel does not fit on an SM");
    }
    choose_tiling(c);
    const int staged_blocks = ((p->nx + 31) / 32) * ((p->ny + 7) / 8);
    c->parts_cap = std::max(c->nitems, staged_blocks);
    if (cudaMalloc(&c->parts, c->parts_cap * sizeof(Part)) != cudaSuccess ||
        cudaMalloc(&c->parts2, c->parts_cap * sizeof(Part)) != cudaSuccess)
        return bail(SWE_ERR_OOM, "partials");
    cudaMemsetAsync(c->parts, 0, c->parts_cap * sizeof(Part), c->st);
    cudaMemsetAsync(c->parts2, 0, c->parts_cap * sizeof(Part), c->st);
    if (p->mode == SWE_STAGED) {
        for (int k = 0; k < SF_COUNT; ++k) {
            if (cudaMalloc(&c->scr[k], c->plane) != cudaSuccess) return bail(SWE_ERR_OOM, "staged intermediates");
            if (cudaMemsetAsync(c->scr[k], 0, c->plane, c->st) != cudaSuccess) return bail(SWE_ERR_CUDA, "memset");
        }
    } else {
        int rc = SWE_OK;
        for (int b = 0; b < 2 && !rc; ++b) {
            rc = encode_map(c, &c->tmH[b], c->f[3 * b]);
            if (!rc) rc = encode_map(c, &c->tmQx[b], c->f[3 * b + 1]);
            if (!rc) rc = encode_map(c, &c->tmQy[b], c->f[3 * b + 2]);
        }
        if (!rc) rc = encode_map(c, &c->tmB, c->f[6]);
        if (!rc) rc = encode_map(c, &c->tmN, c->f[7]);
        for (int b = 0; b < 2 && !rc && c->f[8]; ++b)
            for (int q = 0; q < NACC && !rc; ++q) rc = encode_map(c, &c->tmA[b][q], c->f[8 + NACC * b + q]);
        if (rc) {
            std::string m = g_err;
            return bail(rc, m);
        }
    }
    if (p->skip_dry) {
        // stamps start far in the past: no block is known to be wet
        c->act_nbx = (p->nx + (1 << ACT_LX) - 1) >> ACT_LX;
        c->act_nby = (p->ny + (1 << ACT_LY) - 1) >> ACT_LY;
        const size_t nb = (size_t)c->act_nbx * c->act_nby * sizeof(long long);
        if (cudaMalloc(&c->d_act, nb) != cudaSuccess) return bail(SWE_ERR_OOM, "wet-block stamps");
        if (cudaMemsetAsync(c->d_act, 0x80, nb, c->st) != cudaSuccess) return bail(SWE_ERR_CUDA, "memset");
        if (cudaMalloc(&c->d_hist, c->parts_cap) != cudaSuccess) return bail(SWE_ERR_OOM, "skip history");
        if (cudaMemsetAsync(c->d_hist, 0, c->parts_cap, c->st) != cudaSuccess) return bail(SWE_ERR_CUDA, "memset");
    }
    c->h_b.assign((size_t)p->nx * p->ny, 0.0);
    c->h_solid.assign((size_t)p->nx * p->ny, 0);
    // empty source tables
    c->nsrc = 0;
    int rc = build_source_tables(c, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (rc) {
        std::string m = g_err;
        return bail(rc, m);
    }
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return bail(SWE_ERR_CUDA, "initialisation");
    *out = c;
    return SWE_OK;
}

int swe_set_terrain(swe_ctx* c, const double* b, const double* n) {
    if (!c || !b) return fail(SWE_ERR_ARG, "null argument");
    const size_t N = (size_t)c->p.nx * c->p.ny;
    if (!finite_all(b, N) || (n && !finite_all(n, N))) return fail(SWE_ERR_NONFINITE, "terrain not finite");
    for (size_t k = 0; k < N; ++k)
        if (std::fabs(b[k]) >= 1e20) return fail(SWE_ERR_ARG, "|b| must stay below 1e20");
    CK(cudaSetDevice(c->dev));
    int rc = upload_field(c, b, c->f[6]);
    if (!rc && n) rc = upload_field(c, n, c->f[7]);
    if (!rc && !n) CK(cudaMemsetAsync(c->f[7], 0, c->plane, c->st));
    if (rc) return rc;
    // keep the host copy before re-closing gates over it
    CK(cudaStreamSynchronize(c->st));
    std::memcpy(c->h_b.data(), b, N * sizeof(double));
    std::vector<int> closed;
    for (size_t k = 0; k < N; ++k)
        if (c->h_solid[k]) closed.push_back((int)k);
    rc = apply_beds(c, closed);
    if (rc) return rc;
    if (c->has_state) return state_speed(c);
    return SWE_OK;
}

int swe_set_terrain_ext(swe_ctx* c, const double* b, const double* n) {
    if (!c || !b) return fail(SWE_ERR_ARG, "null argument");
    if (!c->p.ghost_ring) return fail(SWE_ERR_STATE, "swe_set_terrain_ext needs a ghost_ring context");
    const int nxe = c->p.nx + 2 * PAD, nye = c->p.ny + 2 * PAD;
    const size_t N = (size_t)nxe * nye;
    if (!finite_all(b, N) || (n && !finite_all(n, N))) return fail(SWE_ERR_NONFINITE, "terrain not finite");
    for (int j = 0; j < nye; ++j)
        for (int i = 0; i < nxe; ++i) {
            const bool inner = i >= PAD && i < PAD + c->p.nx && j >= PAD && j < PAD + c->p.ny;
            const double v = b[(size_t)j * nxe + i];
            if (inner ? std::fabs(v) >= 1e20 : (std::fabs(v) >= 1e20 && v < 1e29))
                return fail(SWE_ERR_ARG, "|b| must stay below 1e20 (ring cells may be walls, b >= 1e29)");
        }
    CK(cudaSetDevice(c->dev));
    int rc = ensure_staging(c, N * sizeof(double));
    if (rc) return rc;
    for (int q = 0; q < 2; ++q) {
        const double* src = q == 0 ? b : n;
        void* dst = c->f[6 + q];
        if (!src) {
            CK(cudaMemsetAsync(dst, 0, c->plane, c->st));
            continue;
        }
        CK(cudaMemcpyAsync(c->staging, src, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
        CK(is64(c) ? launch_pack_full<double>(c->staging, (double*)dst, nxe, nye, c->pitch, c->st)
                   : launch_pack_full<float>(c->staging, (float*)dst, nxe, nye, c->pitch, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    for (int j = 0; j < c->p.ny; ++j)
        std::memcpy(&c->h_b[(size_t)j * c->p.nx], &b[(size_t)(j + PAD) * nxe + PAD], c->p.nx * sizeof(double));
    std::vector<int> closed;
    for (size_t k = 0; k < c->h_solid.size(); ++k)
        if (c->h_solid[k]) closed.push_back((int)k);
    rc = apply_beds(c, closed);
    if (rc) return rc;
    if (c->has_state) return state_speed(c);
    return SWE_OK;
}

int swe_set_state(swe_ctx* c, const double* H, const double* Qx, const double* Qy, double t) {
    if (!c || !H || !Qx || !Qy) return fail(SWE_ERR_ARG, "null argument");
    const double* src[3] = {H, Qx, Qy};
    return set_state_with(c, t, [&](int k, int neg) { return upload_field(c, src[k], c->f[k], &c->ctl->err, neg); });
}

int swe_set_state_native(swe_ctx* c, const void* H, const void* Qx, const void* Qy, double t) {
    if (!c || !H || !Qx || !Qy) return fail(SWE_ERR_ARG, "null argument");
    const void* src[3] = {H, Qx, Qy};
    return set_state_with(c, t, [&](int k, int) { return upload_native(c, src[k], c->f[k]); }, true);
}

int swe_set_sources(swe_ctx* c, int32_t n, const int32_t* ix, const int32_t* iy, const double* w,
                    const double* vx, const double* vy, const int32_t* hy, int32_t nh, const double* tab) {
    if (!c) return fail(SWE_ERR_ARG, "null context");
    if (n < 0 || nh < 0 || nh > MAX_HYDRO) return fail(SWE_ERR_ARG, "source counts out of range");
    if (n > 0 && (!ix || !iy || !w || !hy || !tab || nh < 1)) return fail(SWE_ERR_ARG, "null source array");
    std::vector<int> cells;
    for (int m = 0; m < n; ++m) {
        if (ix[m] < 0 || ix[m] >= c->p.nx || iy[m] < 0 || iy[m] >= c->p.ny) return fail(SWE_ERR_ARG, "source outside grid");
        if (hy[m] < 0 || hy[m] >= nh) return fail(SWE_ERR_ARG, "hydrograph index");
        if (!std::isfinite(w[m]) || (vx && !std::isfinite(vx[m])) || (vy && !std::isfinite(vy[m])))
            return fail(SWE_ERR_NONFINITE, "source values");
        cells.push_back(iy[m] * c->p.nx + ix[m]);
    }
    std::sort(cells.begin(), cells.end());
    if (std::adjacent_find(cells.begin(), cells.end()) != cells.end()) return fail(SWE_ERR_ARG, "duplicate source cell");
    for (int r = 0; r < nh; ++r) {
        const double* row = tab + 4 * r;
        if (!(row[0] == 0.0 || row[0] == 1.0) || !std::isfinite(row[1]) || !std::isfinite(row[2]) ||
            !std::isfinite(row[3]) || (row[0] == 0.0 && !(row[3] > 0.0)))
            return fail(SWE_ERR_ARG, "hydrograph row");
    }
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->st));
    drop_graph(c);
    cudaFree(c->d_scell); cudaFree(c->d_shydro); cudaFree(c->d_sw); cudaFree(c->d_svx); cudaFree(c->d_svy);
    cudaFree(c->d_hydro);
    c->d_scell = nullptr; c->d_shydro = nullptr; c->d_sw = nullptr; c->d_svx = nullptr; c->d_svy = nullptr;
    c->d_hydro = nullptr;
    c->nsrc = n;
    c->nh = nh;
    c->generation++;
    c->hs_ix.assign(ix, ix + n);
    c->hs_iy.assign(iy, iy + n);
    c->hs_hy.assign(hy, hy + n);
    c->hs_w.assign(w, w + n);
    c->hs_vx.assign(n, 0.0);
    c->hs_vy.assign(n, 0.0);
    if (vx) c->hs_vx.assign(vx, vx + n);
    if (vy) c->hs_vy.assign(vy, vy + n);
    const size_t nn = std::max(1, n);
    if (cudaMalloc(&c->d_scell, nn * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_shydro, nn * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_sw, nn * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_svx, nn * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_svy, nn * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_hydro, std::max(1, nh) * 4 * sizeof(double)) != cudaSuccess)
        return fail(SWE_ERR_OOM, "source allocation");
    if (n > 0) {
        std::vector<int> pc(n);
        std::vector<double> zx(n, 0.0);
        for (int m = 0; m < n; ++m) pc[m] = (iy[m] + PAD) * c->pitch + (ix[m] + PAD);
        CK(cudaMemcpy(c->d_scell, pc.data(), n * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_shydro, hy, n * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_sw, w, n * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_svx, vx ? vx : zx.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_svy, vy ? vy : zx.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_hydro, tab, nh * 4 * sizeof(double), cudaMemcpyHostToDevice));
    }
    return build_source_tables(c, ix, iy, w, vx, vy, hy);
}

int swe_set_solid(swe_ctx* c, int32_t n, const int32_t* ix, const int32_t* iy, const uint8_t* closed) {
    if (!c) return fail(SWE_ERR_ARG, "null context");
    if (n < 0 || (n > 0 && (!ix || !iy || !closed))) return fail(SWE_ERR_ARG, "gate arrays");
    std::vector<int> cells;
    for (int m = 0; m < n; ++m) {
        if (ix[m] < 0 || ix[m] >= c->p.nx || iy[m] < 0 || iy[m] >= c->p.ny) return fail(SWE_ERR_ARG, "gate outside grid");
        if (closed[m] > 1) return fail(SWE_ERR_ARG, "closed must be 0 or 1");
    }
    CK(cudaSetDevice(c->dev));
    for (int m = 0; m < n; ++m) {
        const int k = iy[m] * c->p.nx + ix[m];
        c->h_solid[k] = closed[m];
        cells.push_back(k);
    }
    int rc = apply_beds(c, cells);
    if (rc) return rc;
    if (c->has_state) return state_speed(c);
    return SWE_OK;
}

int swe_step(swe_ctx* c, int32_t nsteps, double t_end, swe_step_info* info) {
    if (!c) return fail(SWE_ERR_ARG, "null context");
    if (nsteps < 0) return fail(SWE_ERR_ARG, "nsteps < 0");
    if (!std::isfinite(t_end)) return fail(SWE_ERR_ARG, "t_end not finite");
    if (!c->has_state) return fail(SWE_ERR_STATE, "swe_set_state has not been called");
    CK(cudaSetDevice(c->dev));
    CK(launch_set_tend(c->ctl, t_end, c->st));
    if (c->p.mode == SWE_STAGED) {
        for (int s = 0; s < nsteps; ++s) {
            if (t_end > 0.0) {
                int rc = read_ctl(c);
                if (rc) return rc;
                if (c->ctl_host->t >= t_end) break;
            }
            int rc = launch_one_step(c);
            if (rc) return rc;
        }
    } else if (nsteps == 1) {
        int rc = launch_one_step(c);
        if (rc) return rc;
    } else if (nsteps > 1) {
        if (!c->gexec || c->gsteps != nsteps) {
            drop_graph(c);
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
            int rc = SWE_OK;
            for (int s = 0; s < nsteps && !rc; ++s) rc = launch_one_step(c);
            cudaError_t e = cudaStreamEndCapture(c->st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return fail(SWE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&c->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(SWE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            c->gsteps = nsteps;
        }
        CK(cudaGraphLaunch(c->gexec, c->st));
    }
    if (info) {
        int rc = read_ctl(c);
        if (rc) return rc;
        const Ctl& h = *c->ctl_host;
        info->t = h.t;
        info->dt_last = h.tau_last;
        info->mass = h.mass;
        info->src_vol = h.src_vol;
        info->clip_vol = h.clip_vol;
        info->max_speed = h.max_speed;
        info->wet_cells = h.wet;
        info->step = h.step;
        info->err_word = (int32_t)h.err;
        info->skipped = (int32_t)h.skipped;
        if (h.err & ERR_TIMEOUT) return fail(SWE_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
        if (h.err & ERR_NONFINITE) return fail(SWE_ERR_NONFINITE, "non-finite signal speed or state");
    }
    return SWE_OK;
}

int swe_get_state(swe_ctx* c, double* H, double* Qx, double* Qy, double* t) {
    if (!c) return fail(SWE_ERR_ARG, "null context");
    if (!c->has_state) return fail(SWE_ERR_STATE, "no state");
    CK(cudaSetDevice(c->dev));
    int rc = read_ctl(c);
    if (rc) return rc;
    const int buf = (int)(c->ctl_host->step & 1);
    double* outs[3] = {H, Qx, Qy};
    for (int k = 0; k < 3 && !rc; ++k)
        if (outs[k]) rc = download_field(c, c->f[3 * buf + k], outs[k], c->p.nx, c->p.ny, 0);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->st));
    if (t) *t = c->ctl_host->t;
    return SWE_OK;
}

int swe_get_state_native(swe_ctx* c, void* H, void* Qx, void* Qy, double* t) {
    if (!c) return fail(SWE_ERR_ARG, "null context");
    if (!c->has_state) return fail(SWE_ERR_STATE, "no state");
    CK(cudaSetDevice(c->dev));
    int rc = read_ctl(c);
    if (rc) return rc;
    const int buf = (int)(c->ctl_host->step & 1);
    const size_t row = (size_t)c->p.nx * c->esz;
    const size_t off = ((size_t)PAD * c->pitch + PAD) * c->esz;
    void* outs[3] = {H, Qx, Qy};
    for (int k = 0; k < 3; ++k)
        if (outs[k])
            CK(cudaMemcpy2DAsync(outs[k], row, (const char*)c->f[3 * buf + k] + off, (size_t)c->pitch * c->esz, row,
                                 (size_t)c->p.ny, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (t) *t = c->ctl_host->t;
    return SWE_OK;
}

int swe_get_device_ptrs(swe_ctx* c, void** H, void** Qx, void** Qy, int64_t* pitch, int32_t* esz) {
    if (!c) return fail(SWE_ERR_ARG, "null context");
    CK(cudaSetDevice(c->dev));
    int rc = read_ctl(c);
    if (rc) return rc;
    const int buf = (int)(c->ctl_host->step & 1);
    const size_t off = ((size_t)PAD * c->pitch + PAD) * c->esz;
    if (H) *H = (char*)c->f[3 * buf + 0] + off;
    if (Qx) *Qx = (char*)c->f[3 * buf + 1] + off;
    if (Qy) *Qy = (char*)c->f[3 * buf + 2] + off;
    if (pitch) *pitch = c->pitch;
    if (esz) *esz = c->esz;
    return SWE_OK;
}

int swe_get_stages(swe_ctx* c, double* const* out) {
    if (!c || !out) return fail(SWE_ERR_ARG, "null argument");
    if (c->p.mode != SWE_STAGED) return fail(SWE_ERR_STATE, "context is not in SWE_STAGED mode");
    CK(cudaSetDevice(c->dev));
    const int nx = c->p.nx, ny = c->p.ny;
    int rc = ensure_staging(c, (size_t)(nx + 1) * (ny + 1) * sizeof(double));
    if (rc) return rc;
    // cell fields in the order of the header, then the face fluxes
    const int order[20] = {SF_UX, SF_UY, SF_AX, SF_AY, SF_PHI, SF_USX, SF_USY, SF_HS, SF_AX2, SF_AY2,
                           SF_PHI2, SF_UTX, SF_UTY, SF_UHX, SF_UHY, SF_HT, SF_QTX, SF_QTY, SF_UPX, SF_UPY};
    for (int k = 0; k < 20 && !rc; ++k)
        if (out[k]) rc = download_field(c, c->scr[order[k]], out[k], nx, ny, 0);
    for (int q = 0; q < 3 && !rc; ++q) {
        if (out[20]) rc = download_field(c, c->scr[SF_FX0 + q], out[20] + (size_t)q * ny * (nx + 1), nx + 1, ny, -1);
        if (!rc && out[21])
            rc = download_field(c, c->scr[SF_FY0 + q], out[21] + (size_t)q * (ny + 1) * nx, nx, ny + 1,
                                -(long long)c->pitch);
        if (!rc) CK(cudaStreamSynchronize(c->st));
    }
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->st));
    return SWE_OK;
}

int swe_sync(swe_ctx* c) {
    if (!c) return fail(SWE_ERR_ARG, "null context");
    CK(cudaStreamSynchronize(c->st));
    return SWE_OK;
}

int swe_autotune(swe_ctx* c, int32_t trial_steps, int32_t* seg_h_out) {
    if (!c || trial_steps < 1) return fail(SWE_ERR_ARG, "null context or trial_steps < 1");
    if (c->p.mode != SWE_FUSED) return fail(SWE_ERR_STATE, "autotuning applies to SWE_FUSED contexts");
    if (!c->has_state) return fail(SWE_ERR_STATE, "swe_set_state has not been called");
    CK(cudaSetDevice(c->dev));
    Snapshot sn;
    int rc = snapshot_take(c, sn);
    if (rc) {
        snapshot_free(sn);
        return rc;
    }
    const int saved = c->p.seg_h;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best = c->seg_h;
    for (int cand : kTileCandidates) {
        if (cand > 2 * c->p.ny && cand != kTileCandidates[0]) break;
        rc = retile(c, cand);
        if (!rc) rc = launch_one_step(c);  // warm-up
        if (!rc) rc = snapshot_restore(c, sn);
        if (rc) break;
        cudaEventRecord(e0, c->st);
        for (int s = 0; s < trial_steps && !rc; ++s) rc = launch_one_step(c);
        cudaEventRecord(e1, c->st);
        if (!rc && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        if (!rc) rc = snapshot_restore(c, sn);
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) rc = retile(c, best);
    else retile(c, saved);
    if (!rc) rc = snapshot_restore(c, sn);
    snapshot_free(sn);
    if (!rc && seg_h_out) *seg_h_out = best;
    return rc;
}

int swe_batch_create(swe_ctx* const* ctxs, int32_t n, swe_batch** out) {
    if (!ctxs || !out || n < 1) return fail(SWE_ERR_ARG, "null argument or n < 1");
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!ctxs[k]) return fail(SWE_ERR_ARG, "null context");
        if (ctxs[k]->p.mode != SWE_FUSED) return fail(SWE_ERR_ARG, "batched contexts must be SWE_FUSED");
        if (ctxs[k]->p.ghost_ring) return fail(SWE_ERR_ARG, "batched contexts need wall boundaries (no ghost ring)");
        if (ctxs[k]->p.precision != ctxs[0]->p.precision) return fail(SWE_ERR_ARG, "mixed precisions");
        if (ctxs[k]->dev != ctxs[0]->dev) return fail(SWE_ERR_ARG, "contexts on different devices");
        if (!ctxs[k]->has_state) return fail(SWE_ERR_STATE, "a context has no state");
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == ctxs[k]) return fail(SWE_ERR_ARG, "a context appears twice");
    }
    swe_batch* b = new (std::nothrow) swe_batch();
    if (!b) return fail(SWE_ERR_OOM, "batch");
    b->ctx.assign(ctxs, ctxs + n);
    b->f64 = ctxs[0]->p.precision == SWE_F64;
    b->dev = ctxs[0]->dev;
    b->st = ctxs[0]->st;
    auto bail = [&](int code) {
        std::string m = g_err;
        swe_batch_destroy(b);
        return fail(code, m);
    };
    if (cudaSetDevice(b->dev) != cudaSuccess) return bail(fail(SWE_ERR_CUDA, "cudaSetDevice"));
    int occ = 0;
    cudaError_t e = b->f64 ? prepare_fused_batch<double>(&occ) : prepare_fused_batch<float>(&occ);
    if (e != cudaSuccess || occ < 1) return bail(fail(SWE_ERR_CUDA, "batch kernel setup"));
    b->grid = ctxs[0]->sm_count * occ;
    if (cudaMalloc(&b->bc, sizeof(BatchCtl)) != cudaSuccess) return bail(fail(SWE_ERR_OOM, "batch control"));
    if (cudaMemset(b->bc, 0, sizeof(BatchCtl)) != cudaSuccess) return bail(fail(SWE_ERR_CUDA, "memset"));
    int rc = batch_sync_all(b);
    if (!rc) rc = batch_build(b);
    if (rc) return bail(rc);
    *out = b;
    return SWE_OK;
}

int swe_batch_set_gate_events(swe_batch* b, int32_t n, const int32_t* scen, const int32_t* ix, const int32_t* iy,
                              const int64_t* step, const uint8_t* closed) {
    if (!b || n < 0 || (n > 0 && (!scen || !ix || !iy || !step || !closed))) return fail(SWE_ERR_ARG, "event arrays");
    std::vector<swe_batch::Ev> ev;
    for (int m = 0; m < n; ++m) {
        if (scen[m] < 0 || scen[m] >= (int)b->ctx.size()) return fail(SWE_ERR_ARG, "event scenario");
        swe_ctx* c = b->ctx[scen[m]];
        if (ix[m] < 0 || ix[m] >= c->p.nx || iy[m] < 0 || iy[m] >= c->p.ny) return fail(SWE_ERR_ARG, "event cell");
        if (closed[m] > 1 || step[m] < 0) return fail(SWE_ERR_ARG, "event step or state");
        ev.push_back({(long long)step[m], scen[m], iy[m] * c->p.nx + ix[m], closed[m]});
    }
    std::stable_sort(ev.begin(), ev.end(), [](const swe_batch::Ev& x, const swe_batch::Ev& y) { return x.step < y.step; });
    CK(cudaSetDevice(b->dev));
    int rc = batch_sync_all(b);
    if (rc) return rc;
    batch_drop_graph(b);
    cudaFree(b->d_ev_idx);
    cudaFree(b->d_ev_val);
    b->d_ev_idx = nullptr;
    b->d_ev_val = nullptr;
    b->events = ev;
    if (ev.empty()) return SWE_OK;
    std::vector<int> idx(ev.size());
    std::vector<double> val(ev.size());
    for (size_t m = 0; m < ev.size(); ++m) {
        swe_ctx* c = b->ctx[ev[m].scen];
        const int i = ev[m].cell % c->p.nx, j = ev[m].cell / c->p.nx;
        idx[m] = (j + PAD) * c->pitch + (i + PAD);
        val[m] = ev[m].closed ? WALL_BED : c->h_b[ev[m].cell];
    }
    if (cudaMalloc(&b->d_ev_idx, idx.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_ev_val, val.size() * sizeof(double)) != cudaSuccess)
        return fail(SWE_ERR_OOM, "events");
    CK(cudaMemcpy(b->d_ev_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_ev_val, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice));
    return SWE_OK;
}

int swe_batch_step(swe_batch* b, int32_t nsteps, swe_step_info* infos) {
    if (!b || nsteps < 0) return fail(SWE_ERR_ARG, "null batch or nsteps < 0");
    CK(cudaSetDevice(b->dev));
    int rc = SWE_OK;
    bool stale = false;
    for (size_t k = 0; k < b->ctx.size(); ++k) stale |= b->ctx[k]->generation != b->gen[k];
    rc = batch_sync_all(b);
    if (!rc && stale) rc = batch_build(b);
    if (rc) return rc;
    for (swe_ctx* c : b->ctx) CK(launch_set_tend(c->ctl, 0.0, b->st));
    if (nsteps > 0) {
        // a window without gate events is the same graph at every base step
        const bool has_ev = std::any_of(b->events.begin(), b->events.end(), [&](const swe_batch::Ev& e) {
            return e.step >= b->step && e.step < b->step + nsteps;
        });
        cudaGraphExec_t* slot = nullptr;
        if (!has_ev) {
            slot = &b->plain[nsteps];
        } else {
            if (!(b->gexec && b->gbase == b->step && b->gsteps == nsteps) && b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            slot = &b->gexec;
        }
        if (!*slot) {
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
            for (int s = 0; s < nsteps && !rc; ++s) {
                rc = batch_launch_events(b, b->step + s);
                if (!rc) rc = batch_launch_step(b);
            }
            cudaError_t e = cudaStreamEndCapture(b->st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return fail(SWE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(slot, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(SWE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            if (has_ev) {
                b->gbase = b->step;
                b->gsteps = nsteps;
            }
        }
        CK(cudaGraphLaunch(*slot, b->st));
        // host record of the walls the events have set
        for (const auto& ev : b->events)
            if (ev.step >= b->step && ev.step < b->step + nsteps) b->ctx[ev.scen]->h_solid[ev.cell] = ev.closed;
        b->step += nsteps;
    }
    if (infos) {
        for (size_t k = 0; k < b->ctx.size(); ++k)
            CK(cudaMemcpyAsync(&b->ctx[k]->ctl_host[0], b->ctx[k]->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->st));
        CK(cudaStreamSynchronize(b->st));
        for (size_t k = 0; k < b->ctx.size(); ++k) {
            const Ctl& h = *b->ctx[k]->ctl_host;
            swe_step_info* info = &infos[k];
            info->t = h.t;
            info->dt_last = h.tau_last;
            info->mass = h.mass;
            info->src_vol = h.src_vol;
            info->clip_vol = h.clip_vol;
            info->max_speed = h.max_speed;
            info->wet_cells = h.wet;
            info->step = h.step;
            info->err_word = (int32_t)h.err;
            info->skipped = (int32_t)h.skipped;
            if (h.err & ERR_TIMEOUT) rc = fail(SWE_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
            else if ((h.err & ERR_NONFINITE) && !rc) rc = fail(SWE_ERR_NONFINITE, "non-finite signal speed");
        }
    }
    return rc;
}

int swe_batch_autotune(swe_batch* b, int32_t trial_steps, int32_t* seg_h_out) {
    if (!b || trial_steps < 1) return fail(SWE_ERR_ARG, "null batch or trial_steps < 1");
    CK(cudaSetDevice(b->dev));
    int rc = batch_sync_all(b);
    if (rc) return rc;
    const size_t n = b->ctx.size();
    std::vector<Snapshot> sn(n);
    for (size_t k = 0; k < n && !rc; ++k) rc = snapshot_take(b->ctx[k], sn[k]);
    auto restore_all = [&]() {
        int r = SWE_OK;
        for (size_t k = 0; k < n && !r; ++k) r = snapshot_restore(b->ctx[k], sn[k]);
        return r;
    };
    int maxny = 0;
    for (swe_ctx* c : b->ctx) maxny = std::max(maxny, c->p.ny);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best = kTileCandidates[0];
    for (int cand : kTileCandidates) {
        if (rc) break;
        if (cand > 2 * maxny && cand != kTileCandidates[0]) break;
        for (size_t k = 0; k < n && !rc; ++k) rc = retile(b->ctx[k], cand);
        if (!rc) rc = batch_build(b);
        if (!rc) rc = batch_launch_step(b);
        if (!rc) rc = restore_all();
        if (rc) break;
        cudaEventRecord(e0, b->st);
        for (int s = 0; s < trial_steps && !rc; ++s) rc = batch_launch_step(b);
        cudaEventRecord(e1, b->st);
        if (!rc && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        if (!rc) rc = restore_all();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (size_t k = 0; k < n && !rc; ++k) rc = retile(b->ctx[k], best);
    if (!rc) rc = batch_build(b);
    if (!rc) rc = restore_all();
    for (auto& x : sn) snapshot_free(x);
    if (!rc && seg_h_out) *seg_h_out = best;
    return rc;
}

void swe_batch_destroy(swe_batch* b) {
    if (!b) return;
    cudaSetDevice(b->dev);
    if (b->st) cudaStreamSynchronize(b->st);
    batch_drop_graph(b);
    cudaFree(b->d_descs);
    cudaFree(b->d_work);
    cudaFree(b->bc);
    cudaFree(b->d_ev_idx);
    cudaFree(b->d_ev_val);
    delete b;
}

int swe_restrict_state(swe_ctx* fine, swe_ctx* coarse) {
    if (!fine || !coarse) return fail(SWE_ERR_ARG, "null context");
    if (fine->p.nx != 4 * coarse->p.nx || fine->p.ny != 4 * coarse->p.ny)
        return fail(SWE_ERR_ARG, "the fine grid must be exactly 4x the coarse grid in both directions");
    if (fine->p.precision != coarse->p.precision || fine->dev != coarse->dev)
        return fail(SWE_ERR_ARG, "contexts differ in precision or device");
    if (!fine->has_state) return fail(SWE_ERR_STATE, "the fine context has no state");
    CK(cudaSetDevice(coarse->dev));
    CK(cudaStreamSynchronize(fine->st));
    if (is64(coarse)) CK(launch_restrict<double>(grid_of<double>(fine), fine->ctl, grid_of<double>(coarse), coarse->ctl, coarse->st));
    else CK(launch_restrict<float>(grid_of<float>(fine), fine->ctl, grid_of<float>(coarse), coarse->ctl, coarse->st));
    int rc = state_speed(coarse);
    if (rc) return rc;
    CK(cudaStreamSynchronize(coarse->st));
    coarse->has_state = true;
    return SWE_OK;
}

static int ensure_norm(swe_ctx* c) {
    if (!c->d_norm && cudaMalloc(&c->d_norm, 16 * sizeof(float)) != cudaSuccess) return fail(SWE_ERR_OOM, "norm");
    return SWE_OK;
}

int swe_closure_features(swe_ctx* c, const float* norm_in, void* x) {
    if (!c || !norm_in || !x) return fail(SWE_ERR_ARG, "null argument");
    if (!c->has_state) return fail(SWE_ERR_STATE, "no state");
    for (int k = 0; k < 5; ++k)
        if (!(norm_in[5 + k] > 0.f) || !std::isfinite(norm_in[k])) return fail(SWE_ERR_ARG, "normalisation");
    CK(cudaSetDevice(c->dev));
    float* d = nullptr;
    CK(cudaMalloc(&d, 10 * sizeof(float)));
    CK(cudaMemcpyAsync(d, norm_in, 10 * sizeof(float), cudaMemcpyHostToDevice, c->st));
    cudaError_t e = is64(c) ? launch_features<double>(grid_of<double>(c), c->ctl, (double)c->p.eps_dry, d, x, c->st)
                            : launch_features<float>(grid_of<float>(c), c->ctl, (float)c->p.eps_dry, d, x, c->st);
    cudaError_t e2 = cudaStreamSynchronize(c->st);
    cudaFree(d);
    CK(e);
    CK(e2);
    return SWE_OK;
}

int swe_closure_targets(swe_ctx* pred, swe_ctx* ref, const float* norm_out, float* t) {
    if (!pred || !ref || !norm_out || !t) return fail(SWE_ERR_ARG, "null argument");
    if (pred->p.nx != ref->p.nx || pred->p.ny != ref->p.ny || pred->p.precision != ref->p.precision)
        return fail(SWE_ERR_ARG, "contexts differ in size or precision");
    for (int k = 0; k < 3; ++k)
        if (!(norm_out[3 + k] > 0.f) || !std::isfinite(norm_out[k])) return fail(SWE_ERR_ARG, "normalisation");
    CK(cudaSetDevice(pred->dev));
    CK(cudaStreamSynchronize(ref->st));
    float* d = nullptr;
    CK(cudaMalloc(&d, 6 * sizeof(float)));
    CK(cudaMemcpyAsync(d, norm_out, 6 * sizeof(float), cudaMemcpyHostToDevice, pred->st));
    cudaError_t e = is64(pred) ? launch_targets<double>(grid_of<double>(pred), pred->ctl, grid_of<double>(ref), ref->ctl,
                                                        pred->p.dx, pred->p.eps_dry, d, t, pred->st)
                               : launch_targets<float>(grid_of<float>(pred), pred->ctl, grid_of<float>(ref), ref->ctl,
                                                       pred->p.dx, pred->p.eps_dry, d, t, pred->st);
    cudaError_t e2 = cudaStreamSynchronize(pred->st);
    cudaFree(d);
    CK(e);
    CK(e2);
    return SWE_OK;
}

int swe_closure_bound(swe_ctx* c, double beta) {
    if (!c) return fail(SWE_ERR_ARG, "null context");
    if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(SWE_ERR_ARG, "bound must be finite and >= 0");
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->st));
    if (c->cexec) {  // the bound is a launch argument of the captured steps
        cudaGraphExecDestroy(c->cexec);
        c->cexec = nullptr;
        c->csteps = 0;
    }
    c->corr_bound = beta;
    return SWE_OK;
}

int swe_closure_attach(swe_ctx* c, swe_cnn* cnn, const float* norm) {
    if (!c || !norm) return fail(SWE_ERR_ARG, "null argument");
    if (c->p.mode != SWE_FUSED) return fail(SWE_ERR_ARG, "the closure runs on SWE_FUSED contexts");
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->st));
    if (c->cexec) {
        cudaGraphExecDestroy(c->cexec);
        c->cexec = nullptr;
        c->csteps = 0;
    }
    if (!cnn) {
        c->cnn = nullptr;
        return SWE_OK;
    }
    int n, h, w;
    cnn_shape(cnn, &n, &h, &w);
    if (n != 1 || h != c->p.ny || w != c->p.nx) return fail(SWE_ERR_ARG, "the network's batch shape must be (1, ny, nx)");
    for (int k = 0; k < 5; ++k)
        if (!(norm[5 + k] > 0.f)) return fail(SWE_ERR_ARG, "normalisation");
    // an output spread of 0 (with mean 0) switches that correction off
    for (int k = 0; k < 3; ++k)
        if (!(norm[13 + k] >= 0.f) || !std::isfinite(norm[13 + k]) || !std::isfinite(norm[10 + k]))
            return fail(SWE_ERR_ARG, "normalisation");
    int rc = ensure_norm(c);
    if (rc) return rc;
    if (!c->d_feat && cudaMalloc(&c->d_feat, (size_t)c->p.nx * c->p.ny * 16 * 2) != cudaSuccess)
        return fail(SWE_ERR_OOM, "closure features");
    if (!c->d_corr) {
        if (cudaMalloc(&c->d_corr, 3 * c->plane) != cudaSuccess) return fail(SWE_ERR_OOM, "closure corrections");
        CK(cudaMemsetAsync(c->d_corr, 0, 3 * c->plane, c->st));
    }
    if (!c->d_acc && cudaMalloc(&c->d_acc, 2 * sizeof(double)) != cudaSuccess) return fail(SWE_ERR_OOM, "closure scratch");
    CK(cudaMemcpyAsync(c->d_norm, norm, 16 * sizeof(float), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->cnn = cnn;
    return SWE_OK;
}

int swe_step_closed(swe_ctx* c, int32_t nsteps, swe_step_info* info) {
    if (!c || nsteps < 0) return fail(SWE_ERR_ARG, "null context or nsteps < 0");
    if (!c->cnn) return fail(SWE_ERR_STATE, "no closure network attached");
    if (!c->has_state) return fail(SWE_ERR_STATE, "no state");
    CK(cudaSetDevice(c->dev));
    CK(launch_set_tend(c->ctl, 0.0, c->st));
    int rc = SWE_OK;
    if (nsteps == 1) {
        rc = launch_closed_step(c);
    } else if (nsteps > 1) {
        if (!c->cexec || c->csteps != nsteps) {
            if (c->cexec) cudaGraphExecDestroy(c->cexec);
            c->cexec = nullptr;
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
            for (int s = 0; s < nsteps && !rc; ++s) rc = launch_closed_step(c);
            cudaError_t e = cudaStreamEndCapture(c->st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return fail(SWE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&c->cexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(SWE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            c->csteps = nsteps;
        }
        CK(cudaGraphLaunch(c->cexec, c->st));
    }
    if (rc) return rc;
    if (info) return swe_step(c, 0, 0.0, info);
    return SWE_OK;
}

void swe_destroy(swe_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->st) cudaStreamSynchronize(c->st);
    drop_graph(c);
    for (void* q : c->f) cudaFree(q);
    for (void* q : c->scr) cudaFree(q);
    cudaFree(c->ctl);
    if (c->ctl_host) cudaFreeHost(c->ctl_host);
    cudaFree(c->parts);
    cudaFree(c->parts2);
    cudaFree(c->d_scell); cudaFree(c->d_shydro); cudaFree(c->d_sw); cudaFree(c->d_svx); cudaFree(c->d_svy);
    cudaFree(c->d_hydro);
    cudaFree(c->d_entries);
    cudaFree(c->d_src_off);
    cudaFree(c->staging);
    cudaFree(c->d_tmp_i);
    cudaFree(c->d_tmp_d);
    if (c->cexec) cudaGraphExecDestroy(c->cexec);
    cudaFree(c->d_norm);
    cudaFree(c->d_feat);
    cudaFree(c->d_corr);
    cudaFree(c->d_acc);
    cudaFree(c->d_act);
    cudaFree(c->d_hist);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

// ------------------------------------------------------------------ nesting

struct swe_nest {
    swe_ctx* c = nullptr;  // coarse parent
    swe_ctx* f = nullptr;  // fine patch (ghost ring)
    int ix0 = 0, iy0 = 0;
    cudaEvent_t ev_c = nullptr, ev_f = nullptr;
};

void swe_nest_destroy(swe_nest* n) {
    if (!n) return;
    if (n->c) cudaStreamSynchronize(n->c->st);
    if (n->f) cudaStreamSynchronize(n->f->st);
    if (n->ev_c) cudaEventDestroy(n->ev_c);
    if (n->ev_f) cudaEventDestroy(n->ev_f);
    delete n;
}

int swe_nest_create(swe_ctx* c, swe_ctx* f, int32_t ix0, int32_t iy0, swe_nest** out) {
    if (!c || !f || !out || c == f) return fail(SWE_ERR_ARG, "two distinct contexts and an output pointer needed");
    *out = nullptr;
    if (c->p.mode != SWE_FUSED || f->p.mode != SWE_FUSED) return fail(SWE_ERR_ARG, "nested contexts must be SWE_FUSED");
    if (c->p.precision != f->p.precision) return fail(SWE_ERR_ARG, "nested contexts must share the precision");
    if (f->p.ghost_ring != 1 || c->p.ghost_ring) return fail(SWE_ERR_ARG, "the fine context needs ghost_ring = 1, the coarse 0");
    if (f->p.nx % 4 || f->p.ny % 4) return fail(SWE_ERR_ARG, "fine nx and ny must be multiples of 4");
    if (std::fabs(c->p.dx - 4.0 * f->p.dx) > 1e-12 * c->p.dx) return fail(SWE_ERR_ARG, "fine dx must be coarse dx / 4");
    if (!(c->p.dt_fixed > 0.0) || std::fabs(f->p.dt_fixed - 0.25 * c->p.dt_fixed) > 1e-12 * c->p.dt_fixed)
        return fail(SWE_ERR_ARG, "fixed steps needed: fine dt_fixed = coarse dt_fixed / 4");
    if (ix0 < 3 || iy0 < 3 || ix0 + f->p.nx / 4 + 3 > c->p.nx || iy0 + f->p.ny / 4 + 3 > c->p.ny)
        return fail(SWE_ERR_ARG, "the patch and 3 coarse cells around it must lie inside the coarse grid");
    if (c->dev != f->dev) return fail(SWE_ERR_ARG, "nested contexts must be on one device");
    if (!c->has_state || !f->has_state) return fail(SWE_ERR_STATE, "both contexts need a state");
    CK(cudaSetDevice(c->dev));
    int rc = read_ctl(c);
    if (!rc) rc = read_ctl(f);
    if (rc) return rc;
    const double tc = c->ctl_host->t, tf = f->ctl_host->t;
    if (std::fabs(tc - tf) > 1e-9 * std::max(1.0, std::fabs(tc))) return fail(SWE_ERR_STATE, "the two states are at different times");
    swe_nest* n = new (std::nothrow) swe_nest();
    if (!n) return fail(SWE_ERR_OOM, "nest");
    n->c = c;
    n->f = f;
    n->ix0 = ix0;
    n->iy0 = iy0;
    if (cudaEventCreateWithFlags(&n->ev_c, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&n->ev_f, cudaEventDisableTiming) != cudaSuccess) {
        swe_nest_destroy(n);
        return fail(SWE_ERR_CUDA, "events");
    }
    *out = n;
    return SWE_OK;
}

int swe_nest_step(swe_nest* n, int32_t ncoarse, swe_step_info* info_c, swe_step_info* info_f) {
    if (!n || ncoarse < 0) return fail(SWE_ERR_ARG, "null nest or ncoarse < 0");
    swe_ctx *c = n->c, *f = n->f;
    CK(cudaSetDevice(c->dev));
    const bool d = is64(c);
    for (int k = 0; k < ncoarse; ++k) {
        int rc = swe_step(c, 1, 0.0, nullptr);
        if (rc) return rc;
        CK(cudaEventRecord(n->ev_c, c->st));
        CK(cudaStreamWaitEvent(f->st, n->ev_c, 0));
        for (int s = 0; s < 4; ++s) {
            const double w = 0.25 * s;
            CK(d ? launch_nest_ring<double>(grid_of<double>(f), f->ctl, grid_of<double>(c), c->ctl, n->ix0, n->iy0, w,
                                            f->p.eps_dry, f->st)
                 : launch_nest_ring<float>(grid_of<float>(f), f->ctl, grid_of<float>(c), c->ctl, n->ix0, n->iy0, w,
                                           (double)(float)f->p.eps_dry, f->st));
            CK(d ? launch_band_acc<double>(staged_args<double>(f), f->st)
                 : launch_band_acc<float>(staged_args<float>(f), f->st));
            rc = swe_step(f, 1, 0.0, nullptr);
            if (rc) return rc;
        }
        CK(cudaEventRecord(n->ev_f, f->st));
        CK(cudaStreamWaitEvent(c->st, n->ev_f, 0));
        CK(d ? launch_nest_restrict<double>(grid_of<double>(f), f->ctl, grid_of<double>(c), c->ctl, n->ix0, n->iy0, c->st)
             : launch_nest_restrict<float>(grid_of<float>(f), f->ctl, grid_of<float>(c), c->ctl, n->ix0, n->iy0, c->st));
        // the coarse state changed under the patch: speed and stored
        // accelerations of those cells and their neighbours
        const int i0 = n->ix0 - 1, j0 = n->iy0 - 1, ni = f->p.nx / 4 + 2, nj = f->p.ny / 4 + 2;
        CK(d ? launch_state_speed_region<double>(staged_args<double>(c), i0, j0, ni, nj, c->st)
             : launch_state_speed_region<float>(staged_args<float>(c), i0, j0, ni, nj, c->st));
    }
    int rc = SWE_OK;
    // exact mass, wet cells and speed of the coarse state for the report
    if (info_c && ncoarse > 0) rc = state_speed(c);
    if (!rc && info_c) rc = swe_step(c, 0, 0.0, info_c);
    if (!rc && info_f) rc = swe_step(f, 0, 0.0, info_f);
    if (!rc && !info_c && !info_f) {
        // the next call may change either context from the host
        CK(cudaEventRecord(n->ev_c, c->st));
        CK(cudaStreamWaitEvent(f->st, n->ev_c, 0));
    }
    return rc;
}

int swe_check_bounded_wait(int32_t limit_ms) {
    if (limit_ms < 1 || limit_ms > 2000) return fail(SWE_ERR_ARG, "limit_ms must be in [1, 2000]");
    unsigned* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) return fail(SWE_ERR_OOM, "probe word");
    unsigned h = 0;
    cudaError_t e = cudaMemset(d, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 32>>>(d, (unsigned long long)limit_ms * 1000000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(SWE_ERR_CUDA, cudaGetErrorString(e));
    if (h & ERR_TIMEOUT) return fail(SWE_ERR_DEVICE_TIMEOUT, "the probe's bounded wait ran out, as it must");
    return SWE_OK;
}

}  // extern "C"
