// bf_execute_noalloc: Algorithm 2 on one image without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// real-time video or imaging pipeline that reserves all of its GPU memory at
// start-up (so that no frame ever waits on the allocator or risks running
// out mid-stream), or a host application that owns the device's memory
// budget and only lends this library the image buffers.  Such callers
// cannot create a plan, because bf_plan allocates the plan's workspace.
// This entry point serves them: the caller passes only the input and output
// images, and every piece of scratch the three kernels need (the T word, the
// parameter set and pair table, the spatial taps, the log-factorial table,
// the status and guard counters) lives in one file-scope static __device__
// array of fixed size, kNoAllocBytes, that every GPU loading the library
// holds until the process exits.
//
// The scratch is filled by a small set-up kernel at the start of every call:
// the spatial taps and the log(k!) table are computed on the host, with the
// same host exp and lgamma as bf_plan, and reach the device as that kernel's
// parameters (no host-to-device copy, no staging buffer), so N, M and the
// weights equal a plan's; T and the counters are cleared.  The status word
// is cleared by bf_noalloc_device_status, which reads it.  Calls share the
// array: two calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on it and must be
// serialised by the caller.
#include <math.h>
#include <mutex>

#include "bf_internal.cuh"

namespace {

using namespace bf;

constexpr int kNoAllocMaxN = 1024;   // largest order N the pair table holds
constexpr int kNoAllocMaxR = 48;     // largest radius R = ceil(3 sigma_s)
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    unsigned Tbits;
    unsigned status;
    unsigned long long n_guarded;
    unsigned pad[4];
    SetHdr hdr;
    float taps[2 * kNoAllocMaxR + 1 + 3];
    double logfact[kNoAllocMaxN + 1];
    Pair pairs[kNoAllocMaxN / 2 + 1];
};
constexpr size_t kNoAllocBytes = (sizeof(NoAllocScratch) + 255) / 256 * 256;

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_addr_mu;
NoAllocScratch* g_addr[kMaxDevices];

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
cudaError_t scratch_on_current_device(NoAllocScratch** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Host-computed tables for one call, passed by value as the set-up kernel's
// parameter (about 8.6 KB, within the 32 KB parameter space of sm_70 and up).
struct NoAllocTables {
    float taps[2 * kNoAllocMaxR + 1 + 3];
    double logfact[kNoAllocMaxN + 1];
};

__global__ void k_noalloc_setup(NoAllocScratch* s, const __grid_constant__ NoAllocTables t, int R,
                                int n_cap)
{
    if (threadIdx.x == 0) {
        s->Tbits = 0u;
        s->n_guarded = 0ull;
    }
    for (int k = threadIdx.x; k <= 2 * R; k += blockDim.x) s->taps[k] = t.taps[k];
    for (int k = threadIdx.x; k <= n_cap; k += blockDim.x) s->logfact[k] = t.logfact[k];
}

int order_bound(double T, double sigma_r)
{
    const double kPi = 3.14159265358979323846;
    const double n0 = (4.0 * T * T) / (kPi * kPi * sigma_r * sigma_r);
    const double c = ceil(n0);
    if (c < 1.0) return 1;
    if (c > 1e9) return 1000000000;
    return (int)c;
}

}  // namespace

extern "C" bf_status bf_execute_noalloc(const float* f, size_t f_pitch, float* out,
                                        size_t out_pitch, int H, int W, double sigma_s,
                                        double sigma_r, double eps, float value_range,
                                        void* stream)
{
    if (!f || !out || (const void*)f == (const void*)out) return BF_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || H > (1 << 16) || W > (1 << 16)) return BF_ERR_INVALID_ARG;
    if (f_pitch < (size_t)W || out_pitch < (size_t)W) return BF_ERR_INVALID_ARG;
    if (!(sigma_s > 0.0) || !(sigma_r > 0.0) || !(eps >= 0.0) || !(eps < 1.0))
        return BF_ERR_INVALID_ARG;
    if (!isfinite(sigma_s) || !isfinite(sigma_r) || !(value_range > 0.f) || !isfinite(value_range))
        return BF_ERR_INVALID_ARG;
    const double Rr = ceil(3.0 * sigma_s);
    if (Rr > (double)kNoAllocMaxR) return BF_ERR_NOT_SUPPORTED;   // radius above the scratch size
    const int R = (int)Rr;
    int th = 0, tw = 0;
    fwd32_tile(R, &th, &tw);
    if (!th || R > range_max_radius()) return BF_ERR_NOT_SUPPORTED;
    // the largest N an image within [0, value_range] can need must fit the table
    const int n_cap = order_bound((double)value_range, sigma_r);
    if (n_cap > kNoAllocMaxN) return BF_ERR_ORDER_TOO_LARGE;

    NoAllocScratch* s = nullptr;
    if (scratch_on_current_device(&s) != cudaSuccess) return BF_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;

    // taps g(k) = exp(-k^2 / (2 sigma_s^2)) and log(k!) as bf_plan makes them
    NoAllocTables tab;
    for (int k = -R; k <= R; ++k)
        tab.taps[k + R] = (float)exp(-(double)k * (double)k / (2.0 * sigma_s * sigma_s));
    for (int k = 0; k <= n_cap; ++k) tab.logfact[k] = lgamma((double)k + 1.0);
    k_noalloc_setup<<<1, 256, 0, st>>>(s, tab, R, n_cap);
    if (cudaGetLastError() != cudaSuccess) return BF_ERR_CUDA;
    if (launch_local_range(f, f_pitch, H, W, R, 0, 1, &s->Tbits, st) != cudaSuccess)
        return BF_ERR_CUDA;
    ParamsArgs pa;
    pa.T = reinterpret_cast<const float*>(&s->Tbits);
    pa.n_sets = 1;
    pa.sigma_r = sigma_r;
    pa.eps = eps;
    pa.value_range = value_range;
    pa.rule = BF_RULE_ALG2;
    pa.n_cap = n_cap;
    pa.cap_pairs = n_cap / 2 + 1;
    pa.logfact = s->logfact;
    pa.ln2 = log(2.0);
    pa.hdr = &s->hdr;
    pa.pairs = s->pairs;
    pa.status = &s->status;
    if (launch_params(pa, st) != cudaSuccess) return BF_ERR_CUDA;
    FwdArgs fa;
    fa.f = f;
    fa.f_pitch = f_pitch;
    fa.out = out;
    fa.out_pitch = out_pitch;
    fa.H = H;
    fa.W = W;
    fa.R = R;
    fa.taps = s->taps;
    fa.hdr = &s->hdr;
    fa.pairs = s->pairs;
    fa.cap_pairs = n_cap / 2 + 1;
    fa.set_tile = 0;
    fa.sets_x = 1;
    fa.c0 = 0.5f * value_range;
    fa.n_guarded = &s->n_guarded;
    fa.den_out = nullptr;
    fa.den_pitch = 0;
    // the same taps on the host, for the kernels that take them as a parameter
    fa.h_taps = tab.taps;
    fa.sep_P = nullptr;             // no workspace: the fused tiles serve every radius
    fa.sep_nd = nullptr;
    fa.sep_nk = fa.sep_Wp = fa.sep_cap_terms = 0;
    if (launch_fwd32(fa, st) != cudaSuccess) return BF_ERR_CUDA;
    return BF_OK;
}

// Reads, then clears, the status word the calls on `stream`'s device have
// left in the static scratch (BF_DEV_* bits), after synchronising `stream`.
extern "C" bf_status bf_noalloc_device_status(void* stream, unsigned* bits)
{
    NoAllocScratch* s = nullptr;
    if (scratch_on_current_device(&s) != cudaSuccess) return BF_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned v = 0;
    if (cudaMemcpyAsync(&v, &s->status, sizeof(v), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BF_ERR_CUDA;
    if (cudaMemsetAsync(&s->status, 0, sizeof(unsigned), st) != cudaSuccess) return BF_ERR_CUDA;
    if (bits) *bits = v;
    return v ? BF_ERR_DEVICE_STATUS : BF_OK;
}
