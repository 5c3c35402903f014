// swe_step_f32_noalloc: one fused FP32 time step on caller-owned device
// planes that allocates no device memory at all.
//
// Who needs it: callers that cannot call cudaMalloc themselves or through
// this library -- code that gets all of its device memory from a host
// framework's own pool or arena, code with a fixed device-memory budget, or
// loops that must not call cudaMalloc/cudaFree because those calls can
// synchronise the whole device.  They pass the state, statics and outputs;
// the only other global memory the fused kernel needs (its control block,
// one partial-sum record per CTA and an empty source table) lives in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/swe.h"
#include "swe_launch.h"

using namespace swe;

namespace {

// Layout of the scratch array: [Ctl | src_off (items + 1 ints) | Part x items]
constexpr size_t kCtlBytes = 256;
constexpr size_t kOffBytes = ((size_t)(SWE_NOALLOC_MAX_ITEMS + 1) * sizeof(int) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCtlBytes + kOffBytes + (size_t)SWE_NOALLOC_MAX_ITEMS * sizeof(Part);
static_assert(sizeof(Ctl) <= kCtlBytes, "control block does not fit");
static_assert(kScratchBytes == SWE_NOALLOC_SCRATCH_BYTES, "header states a different scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

int nfail(int code, const std::string& m) {
    set_last_error(m.c_str());
    return code;
}

// Clear what must start at zero and set the step's inputs.  The array keeps
// the previous call's contents otherwise.
__global__ void k_noalloc_init(double t, unsigned long long smax_bits, int nitems) {
    Ctl* ctl = reinterpret_cast<Ctl*>(g_noalloc_scratch);
    int* off = reinterpret_cast<int*>(g_noalloc_scratch + kCtlBytes);
    for (int i = threadIdx.x; i <= nitems; i += blockDim.x) off[i] = 0;
    if (threadIdx.x == 0) {
        memset(ctl, 0, sizeof(Ctl));
        ctl->t = t;
        ctl->smax[0] = smax_bits;
        ctl->smax[1] = 0ull;
    }
}

struct DevScratch {
    unsigned char* base = nullptr;
    int occ = 0;
    int sms = 0;
};

std::mutex g_mu;
DevScratch g_dev[64];

// Once per device, with that device current: the device address of the
// scratch array (host code may not use the array's name as an address) and
// the fused kernel's shared-memory opt-in.
int setup_device(int dev, DevScratch** out) {
    if (dev < 0 || dev >= 64) return nfail(SWE_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    DevScratch& d = g_dev[dev];
    if (!d.base) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return nfail(SWE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        e = prepare_fused<float>(&d.occ);
        if (e != cudaSuccess) return nfail(SWE_ERR_CUDA, std::string("fused kernel setup: ") + cudaGetErrorString(e));
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return nfail(SWE_ERR_CUDA, std::string("device attribute: ") + cudaGetErrorString(e));
        d.base = static_cast<unsigned char*>(p);
    }
    *out = &d;
    return SWE_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once (under the set-up mutex).
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
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

int encode(CUtensorMap* m, const void* base, int nx, int ny, int64_t pitch) {
    const EncodeTiledFn fn = encode_fn();
    if (!fn) return nfail(SWE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {(cuuint64_t)(nx + 2 * PAD), (cuuint64_t)(ny + 2 * PAD)};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)WIN, (cuuint32_t)RB};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nfail(SWE_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return SWE_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" SWE_API int swe_step_f32_noalloc(const swe_params* p, const float* H, const float* Qx, const float* Qy,
                                           const float* b, const float* n, float* H_out, float* Qx_out,
                                           float* Qy_out, int64_t pitch, double t, double max_speed,
                                           swe_step_info* info) {
    // argument checks come first and touch no device state
    if (!p || !H || !Qx || !Qy || !b || !n || !H_out || !Qx_out || !Qy_out)
        return nfail(SWE_ERR_ARG, "null argument");
    if (p->precision != SWE_F32) return nfail(SWE_ERR_ARG, "swe_step_f32_noalloc takes FP32 planes only");
    if (p->nx < 1 || p->ny < 1 || p->nx > (1 << 20) || p->ny > (1 << 20))
        return nfail(SWE_ERR_ARG, "grid size out of range");
    if (!(p->dx > 0.0) || !(p->g > 0.0) || !(p->cfl > 0.0 && p->cfl <= 1.0) || !(p->eps_dry >= 0.0) ||
        !(p->dt_max > 0.0) || !(p->dt_fixed >= 0.0) || !(p->nu >= 0.0) || !(p->c_a >= 0.0))
        return nfail(SWE_ERR_ARG, "physical or numerical parameter out of range");
    if (!(p->rain_rate >= 0.0 && p->rain_rate < 1.0) || !(p->evap_rate >= 0.0 && p->evap_rate < 1.0) ||
        !(p->infil_rate >= 0.0 && p->infil_rate < 1.0))
        return nfail(SWE_ERR_ARG, "rain, evaporation and infiltration rates must lie in [0, 1) m/s");
    if (pitch < (int64_t)p->nx + 2 * PAD || (pitch % 4) != 0)
        return nfail(SWE_ERR_ARG, "pitch must be >= nx + 2*SWE_PAD and a multiple of 4 floats");
    // the kernel indexes rows with a 32-bit pitch
    if (pitch > (int64_t)INT_MAX) return nfail(SWE_ERR_ARG, "pitch must not exceed INT_MAX floats");
    const void* ptrs[8] = {H, Qx, Qy, b, n, H_out, Qx_out, Qy_out};
    for (const void* q : ptrs)
        if (!aligned16(q)) return nfail(SWE_ERR_ARG, "every plane must start on a 16-byte boundary");
    if (!(p->dt_fixed > 0.0) && !(max_speed >= 0.0))
        return nfail(SWE_ERR_ARG, "max_speed must be >= 0 unless dt_fixed > 0");
    if (!(t == t) || !(max_speed == max_speed)) return nfail(SWE_ERR_ARG, "t or max_speed is NaN");
    // tiling: the fused kernel's CTAs, each with one partial-sum record
    const int ntx = (p->nx + TW - 1) / TW;
    if (ntx > SWE_NOALLOC_MAX_ITEMS)
        return nfail(SWE_ERR_ARG, "grid too wide for the allocation-free scratch (at most " +
                                      std::to_string(SWE_NOALLOC_MAX_ITEMS) + " CTAs)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(SWE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    DevScratch* d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc) return rc;
    // rows per CTA: fill the GPU once (CTAs per SM x SMs), then grow until
    // the CTA count fits the scratch
    const int slots = d->sms * d->occ;
    int seg_h = (p->ny + std::max(1, slots / ntx) - 1) / std::max(1, slots / ntx);
    seg_h = std::max(seg_h, 16);
    while ((long long)ntx * ((p->ny + seg_h - 1) / seg_h) > SWE_NOALLOC_MAX_ITEMS) seg_h *= 2;
    const int nty = (p->ny + seg_h - 1) / seg_h;
    const int nitems = ntx * nty;

    FusedArgs<float> a;
    std::memset(&a, 0, sizeof(a));
    rc = encode(&a.tmH[0], H, p->nx, p->ny, pitch);
    if (!rc) rc = encode(&a.tmQx[0], Qx, p->nx, p->ny, pitch);
    if (!rc) rc = encode(&a.tmQy[0], Qy, p->nx, p->ny, pitch);
    if (!rc) rc = encode(&a.tmB, b, p->nx, p->ny, pitch);
    if (!rc) rc = encode(&a.tmN, n, p->nx, p->ny, pitch);
    if (rc) return rc;
    a.g.nx = p->nx;
    a.g.ny = p->ny;
    a.g.pitch = (int)pitch;
    a.g.H[0] = const_cast<float*>(H);
    a.g.Qx[0] = const_cast<float*>(Qx);
    a.g.Qy[0] = const_cast<float*>(Qy);
    a.g.H[1] = H_out;
    a.g.Qx[1] = Qx_out;
    a.g.Qy[1] = Qy_out;
    a.g.b = const_cast<float*>(b);
    a.g.n = const_cast<float*>(n);
    a.P.g = (float)p->g;
    a.P.h = (float)p->dx;
    a.P.eps = (float)p->eps_dry;
    a.P.nu = (float)p->nu;
    a.P.f = (float)p->coriolis_f;
    a.P.wx = (float)p->wind_x;
    a.P.wy = (float)p->wind_y;
    a.P.ca = (float)p->c_a;
    a.P.ra = (float)p->rho_air_over_rho;
    a.P.rain = (float)p->rain_rate;
    a.P.loss = (float)(p->evap_rate + p->infil_rate);
    a.P.dist = (p->rain_rate != 0.0 || p->evap_rate != 0.0 || p->infil_rate != 0.0) ? 1 : 0;
    phys_derive(a.P);
    a.sp.dx = p->dx;
    a.sp.cfl = p->cfl;
    a.sp.dt_max = p->dt_max;
    a.sp.dt_fixed = p->dt_fixed;
    a.ctl = reinterpret_cast<Ctl*>(d->base);
    a.src_off = reinterpret_cast<const int*>(d->base + kCtlBytes);
    a.src = reinterpret_cast<const SrcEntry*>(d->base);  // never read: every source list is empty
    a.parts = reinterpret_cast<Part*>(d->base + kCtlBytes + kOffBytes);
    a.hydro = nullptr;
    a.nh = 0;
    a.ntx = ntx;
    a.seg_h = seg_h;
    a.nitems = nitems;

    cudaStream_t st = (cudaStream_t)p->cuda_stream;
    double ms = p->dt_fixed > 0.0 ? 0.0 : max_speed;
    unsigned long long bits;
    std::memcpy(&bits, &ms, sizeof(bits));
    k_noalloc_init<<<1, 256, 0, st>>>(t, bits, nitems);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(SWE_ERR_CUDA, std::string("init launch: ") + cudaGetErrorString(e));
    e = launch_fused<float>(a, st);
    if (e != cudaSuccess) return nfail(SWE_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    if (info) {
        Ctl h;
        e = cudaMemcpyAsync(&h, d->base, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return nfail(SWE_ERR_CUDA, std::string("report copy: ") + cudaGetErrorString(e));
        info->t = h.t;
        info->dt_last = h.tau_last;
        info->mass = h.mass;
        info->src_vol = h.src_vol;
        info->clip_vol = h.clip_vol;
        info->max_speed = h.max_speed;
        info->wet_cells = h.wet;
        info->step = h.step;
        info->err_word = (int32_t)h.err;
        info->skipped = 0;
        if (h.err & ERR_TIMEOUT) return nfail(SWE_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
        if (h.err & ERR_NONFINITE) return nfail(SWE_ERR_NONFINITE, "non-finite signal speed");
        if (h.step != 1) return nfail(SWE_ERR_DT, "time step not positive");
    }
    return SWE_OK;
}
