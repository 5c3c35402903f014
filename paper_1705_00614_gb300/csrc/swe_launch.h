// Types shared by the host API (swe_capi.cu) and the kernel units
// (swe_f32.cu, swe_f64.cu), and the launch functions the kernel units export.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "swe_math.cuh"

struct swe_cnn;

namespace swe {

// Ring of wall cells around every grid (>= the 6-cell dependence radius of
// one fused step; 10 keeps every TMA box start 16-byte aligned).
constexpr int PAD = 10;
// stored accelerations per state buffer: a_x, a_y (the friction coefficient
// is local to the cell and recomputed from the state by the predictor)
constexpr int NACC = 2;
// Fused kernel geometry: a CTA owns a window of WIN columns (one thread per
// column) and streams it down the rows of its segment; HALO columns on each
// side are recomputed, so TW = WIN - 2 HALO columns are produced.
constexpr int WIN = 128;
constexpr int HALO = 6;
constexpr int TW = WIN - 2 * HALO;
constexpr int RB = 1;      // rows per TMA chunk
constexpr int ACT_LX = 5, ACT_LY = 4;  // wet-block stamps: 32 x 16 cells
constexpr int MAX_HYDRO = 32;

enum ErrBits : unsigned int {
    ERR_NONFINITE = 1u,
    ERR_TIMEOUT = 2u,
};

// Device control block of one grid.
struct Ctl {
    double t;          // time at the start of the next step
    double t_end;      // > 0: clamp
    double tau_last;   // tau of the last completed step
    double mass, src_vol, clip_vol, max_speed;  // report of the last completed step
    long long wet;
    long long step;    // steps since the state was set
    long long skipped; // work items of the last step skipped as dry
    unsigned long long smax[2];  // max signal speed (FP64 bits) for the step of that parity
    unsigned int done;           // CTAs finished in the running step
    unsigned int err;            // ErrBits
};

// Per-CTA partial sums of one step (reduced in a fixed order).
struct Part {
    double mass, src, clip;
    int wet;      // wet cells (at most 116 x 32768 per work item)
    int skipped;  // 1 if the item was skipped as dry
};

// One source cell as seen by one work item (window coordinates).
struct SrcEntry {
    short r, c;     // window row and column
    int hydro;
    double w, vx, vy;
};

// Numerical step parameters (FP64, as the time step is formed in FP64).
struct StepP {
    double dx, cfl, dt_max, dt_fixed;
};

template <class T>
struct Grid {
    int nx, ny, pitch;   // interior size, row pitch in elements
    T* H[2];             // padded arrays, pointing at padded (0, 0)
    T* Qx[2];
    T* Qy[2];
    T* b;
    T* n;
    // accelerations (a_x, a_y, phi) of the state in each buffer, or null
    T* A[2][NACC];
};

template <class T>
struct FusedArgs {
    CUtensorMap tmH[2], tmQx[2], tmQy[2], tmB, tmN;
    CUtensorMap tmA[2][NACC];
    // wet-block stamps (skip_dry) or null: per 32 x 16-cell block of the
    // interior grid, the last step at which the block held a wet cell
    long long* act;
    int act_nbx;
    int skip;  // nonzero: items whose window is dry and sourceless may skip
    // per item, bit 0: skipped in the last step, bit 1: in the one before
    // (both: the output buffer already holds what a skip would write)
    unsigned char* hist;
    Grid<T> g;
    Phys<T> P;
    StepP sp;
    Ctl* ctl;
    Part* parts;
    const SrcEntry* src;
    const int* src_off;   // [nitems + 1]
    const double* hydro;  // [nh][4]
    int nh;
    int ntx, seg_h, nitems;
    // open (zero-gradient) ghost ring: the signal speeds of the outermost
    // interior rows and columns come from the band pass after each fill
    int open_ring;
    // learned closure: corrections of the net face-flux sums (3 padded
    // planes F_H, F_Qx, F_Qy), or null
    const T* corr;
    size_t corr_plane;
    // > 0: each correction is bounded by corr_bound times the magnitude of
    // the cell's plain flux sum it corrects
    T corr_bound;
};

// Control block of a batched launch: the next work-list entry to hand out and
// the CTAs that have run out of work (the last one resets both).
struct BatchCtl {
    unsigned next;
    unsigned exited;
};

template <class T>
struct BatchArgs {
    const FusedArgs<T>* descs;  // one per scenario, in device memory (64-byte aligned)
    const int2* work;           // (scenario, item), largest items first
    int nwork;
    BatchCtl* bc;
};

template <class T>
struct StagedArgs {
    Grid<T> g;
    Phys<T> P;
    StepP sp;
    Ctl* ctl;
    Part* parts;
    Part* parts2;
    // intermediates (padded like the state)
    T *ux, *uy, *ax, *ay, *phi, *usx, *usy, *hs, *ax2, *ay2, *phi2;
    T *utx, *uty, *uhx, *uhy, *ht, *qtx, *qty, *upx, *upy;
    T *sig, *svx, *svy;
    T *fx[3], *fy[3];
    // global source list
    const int* s_cell;    // padded linear index
    const int* s_hydro;
    const double* s_w;
    const double* s_vx;
    const double* s_vy;
    int nsrc;
    const double* hydro;
    int nh;
    long long* act;  // wet-block stamps to write for the state, or null
    int act_nbx;
    unsigned char* hist;  // per-item skip history to clear, or null
    int nhist;
    int open_ring;  // as in FusedArgs
};

template <class T>
cudaError_t prepare_fused(int* ctas_per_sm);
template <class T>
cudaError_t prepare_fused_batch(int* ctas_per_sm);
template <class T>
cudaError_t launch_fused_batch(const BatchArgs<T>& b, int grid, cudaStream_t st);
template <class T>
cudaError_t launch_fused(const FusedArgs<T>& a, cudaStream_t st);
template <class T>
cudaError_t launch_staged(const StagedArgs<T>& a, cudaStream_t st);
// Signal speed and mass of the current state (the first step's K3).
template <class T>
// With check != 0 the pass also checks a state just copied in: non-finite
// H, Qx, Qy set error bit 0, a negative depth bit 1.
cudaError_t launch_state_speed(const StagedArgs<T>& a, cudaStream_t st, int check = 0);
// The same over a region of the grid, without the mass report: the speed
// slot takes the max with the region's (an over-estimate at most).
template <class T>
cudaError_t launch_state_speed_region(const StagedArgs<T>& a, int i0, int j0, int ni, int nj, cudaStream_t st);
// Stored accelerations of the ring band after a ghost-ring fill.
template <class T>
cudaError_t launch_band_acc(const StagedArgs<T>& a, cudaStream_t st);
// FP64 row-major [ny][nx] staging -> padded field of type T, and back.
template <class T>
cudaError_t launch_pack(const double* src, T* dst, int nx, int ny, int pitch, cudaStream_t st,
                       unsigned* flag = nullptr, int check_neg = 0);
template <class T>
cudaError_t launch_unpack(const T* src, double* dst, int nx, int ny, int pitch, cudaStream_t st);
// dst[idx[m]] = val[m]
template <class T>
cudaError_t launch_scatter(T* dst, const int* idx, const double* val, int n, cudaStream_t st);
template <class T>
cudaError_t launch_fill_bed(T* b, int nx, int ny, int pitch, cudaStream_t st);
// FP64 row-major [ny + 2 PAD][nx + 2 PAD] -> the whole padded field.
template <class T>
cudaError_t launch_pack_full(const double* src, T* dst, int nxe, int nye, int pitch, cudaStream_t st);
// Two-level nesting: ghost ring of the fine patch from the coarse grid at
// the fraction w of the last coarse step; 4x4 restriction of the patch onto
// the coarse cells it covers.
template <class T>
cudaError_t launch_nest_ring(const Grid<T>& f, const Ctl* fctl, const Grid<T>& c, const Ctl* cctl, int ix0, int iy0,
                             double w, double eps, cudaStream_t st);
template <class T>
cudaError_t launch_nest_restrict(const Grid<T>& f, const Ctl* fctl, const Grid<T>& c, const Ctl* cctl, int ix0, int iy0,
                                 cudaStream_t st);
// Open boundary: non-wall ring cells take the nearest interior cell's state.
template <class T>
cudaError_t launch_ring_outflow(const Grid<T>& g, const Ctl* ctl, cudaStream_t st);
template <class T>
size_t fused_smem_bytes();
// Learned-closure kernels (swe_cnn.cu).
// Standardised coarse features (H, Ux, Uy, b, n) of the state at step
// parity, BF16 [ny][nx][16]; norm = mu[5], sd[5].
template <class T>
cudaError_t launch_features(const Grid<T>& g, const Ctl* ctl, T eps, const float* norm, void* x, cudaStream_t st);
// CNN output (standardised, FP32 [ny][nx][3]) -> flux-sum corrections in
// padded planes for wet cells, depth correction centred over wet cells;
// norm = mu[3], sd[3]; acc: 2 doubles of scratch.
template <class T>
cudaError_t launch_corrections(const Grid<T>& g, const Ctl* ctl, T eps, const float* y, const float* norm, T* corr,
                               size_t plane, double* acc, cudaStream_t st);
// coarse state (buffer 0) := 4x4 block means of the fine state; coarse
// control block := fine time, step 0.
template <class T>
cudaError_t launch_restrict(const Grid<T>& fine, const Ctl* fctl, const Grid<T>& coarse, Ctl* cctl, cudaStream_t st);
// standardised training targets: ((ref - pred) h / tau - mu) / sd, FP32
// [ny][nx][3]; tau = the predicting grid's last step.
template <class T>
cudaError_t launch_targets(const Grid<T>& pred, const Ctl* pctl, const Grid<T>& ref, const Ctl* rctl, double h,
                           double eps, const float* norm, float* t, cudaStream_t st);
// Forward pass of a closure network on a given stream; output FP32
// [n][h][w][3] in the network's own buffer.
int cnn_forward_on(swe_cnn* c, const void* x, cudaStream_t st);
const float* cnn_output(const swe_cnn* c);
void cnn_shape(const swe_cnn* c, int* n, int* h, int* w);

// The message swe_last_error() returns on the calling thread.
void set_last_error(const char* msg);
// Set the device copy of t_end (kernel argument, so it is stream ordered).
cudaError_t launch_set_tend(Ctl* ctl, double t_end, cudaStream_t st);

}  // namespace swe
