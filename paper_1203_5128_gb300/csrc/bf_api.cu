// C ABI of libbf: plans, Algorithm 2 on the device, status and info.
//
// bf_execute enqueues, on the caller's stream and without host
// synchronisation: K1 (local range -> T, Algorithm 1) unless T is fixed, K2
// (N, M, pair table, Algorithm 2 steps 3-5) and the fused forward K3
// (SHIFTABLE-BF, Sec. 1.2).  K3 reads the term count from device memory, so
// a data-dependent N never round-trips through the host.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bf_internal.cuh"

using namespace bf;

namespace bf {
// Defined in the translation units of the other kernels.
cudaError_t launch_backward(bf_plan_s* p, const float* f, const float* gout, float* gin,
                            size_t pitch, cudaStream_t s);
}



namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxTimed = 4096;
constexpr int kEvPerExec = 5;     // before K1, after K1, K2, K3, recheck

// N of the raised polynomial: max(1, ceil(T^2 / (2 sigma_r^2))) (Sec. 1.3)
int poly_order_of(double T, double sigma_r)
{
    const double c = ceil((T * T) / (2.0 * sigma_r * sigma_r));
    if (c < 1.0) return 1;
    if (c > 1e9) return 1000000000;
    return (int)c;
}

int order_of(double T, double sigma_r)
{
    // same arithmetic as the device (K2): N = max(1, ceil(4 T^2 / (pi^2 sigma_r^2)))
    const double n0 = (4.0 * T * T) / (kPi * kPi * sigma_r * sigma_r);
    const double c = ceil(n0);
    if (c < 1.0) return 1;
    if (c > 1e9) return 1000000000;
    return (int)c;
}

bf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? BF_OK : BF_ERR_CUDA; }

// The box filter's FP32 planes take the exact running-sum kernel where the
// FIR would need its small 16 x 16 tiles (per-T-tile plans at large radii;
// image-wide T takes the two-pass FIR, faster there).
bool box_running_sums(const bf_options& o, int R)
{
    if (o.spatial != BF_SPATIAL_BOX || o.range_kernel != BF_RANGE_COSINE || o.patch_mask ||
        o.plane_dtype != BF_PLANES_FP32 || o.filter == BF_FILTER_YVV || o.t_mode != BF_T_TILE)
        return false;
    int th = 0, tw = 0;
    fwd32_tile(R, &th, &tw);
    return th < 32 && !fwd32t_ok(R, o.t_tile) && box32_rows(R, o.t_tile) > 0;
}

#define BF_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return BF_ERR_CUDA;         \
    } while (0)

void free_plan(bf_plan_s* p)
{
    if (!p) return;
    cudaFree(p->d_T);
    cudaFree(p->d_hdr);
    cudaFree(p->d_pairs);
    cudaFree(p->d_taps);
    free(p->h_taps);
    cudaFree(p->d_logfact);
    cudaFree(p->d_status);
    cudaFree(p->d_nguard);
    cudaFree(p->d_hin);
    cudaFree(p->d_hout);
    cudaFree(p->d_yvv_P);
    cudaFree(p->d_yvv_S);
    cudaFree(p->d_yvv_nd);
    cudaFree(p->d_yvv_mass);
    cudaFree(p->d_sep_P);
    cudaFree(p->d_sep_nd);
    cudaFree(p->d_bwd);
    cudaFree(p->d_fix);
    cudaFree(p->d_fixcnt);
    cudaFree(p->d_fixscan);
    cudaFree(p->d_mm);
    if (p->ev) {
        for (int i = 0; i < kEvPerExec * kMaxTimed; ++i)
            if (p->ev[i]) cudaEventDestroy(p->ev[i]);
        free(p->ev);
    }
    for (int i = 0; i < 5; ++i)
        if (p->hst[i]) cudaStreamDestroy(p->hst[i]);
    if (p->hev) {
        for (int i = 0; i < p->n_hev; ++i)
            if (p->hev[i]) cudaEventDestroy(p->hev[i]);
        free(p->hev);
    }
    free(p);
}

ParamsArgs params_args(bf_plan_s* p)
{
    ParamsArgs a;
    a.T = reinterpret_cast<const float*>(p->d_T);
    a.n_sets = p->n_sets;
    a.sigma_r = p->sigma_r;
    a.eps = p->eps;
    a.value_range = p->opt.value_range;
    a.rule = p->opt.trunc_rule;
    a.n_cap = p->n_cap;
    a.cap_pairs = p->cap_pairs;
    a.logfact = p->d_logfact;
    a.ln2 = log(2.0);
    a.hdr = p->d_hdr;
    a.pairs = p->d_pairs;
    a.status = p->d_status;
    return a;
}

}  // namespace

namespace bf {

ParamsArgs plan_params_args(bf_plan_s* p) { return params_args(p); }

YvvArgs yvv_args(bf_plan_s* p, const float* f, size_t fp, float* out, size_t op)
{
    YvvArgs a;
    a.f = f;
    a.f_pitch = fp;
    a.out = out;
    a.out_pitch = op;
    a.H = p->H;
    a.W = p->W;
    a.c0 = p->c0;
    a.hdr = p->d_hdr;
    a.pairs = p->d_pairs;
    a.G = p->yvv_G;
    a.n_nd = p->yvv_G;
    a.P = p->d_yvv_P;
    a.S = p->d_yvv_S;
    a.nd = p->d_yvv_nd;
    a.mass_y = p->d_yvv_mass;
    a.mass_x = p->d_yvv_mass + p->H;
    a.n_guarded = p->d_nguard;
    yvv_design(p->sigma_s, &a.coef, nullptr);
    const YvvCoef& k = a.coef;
    auto two = [](float v) { return make_float2(v, v); };
    a.coef2 = YvvCoef2{two(k.P0), two(k.Pr), two(k.Pi), two(-k.Pi), two(k.C0), two(k.Cr), two(-k.Ci),
                       two(k.D0), two(k.Dr), two(-k.Di)};
    return a;
}

FwdArgs forward_args(bf_plan_s* p, const float* f, size_t fp, float* out, size_t op)
{
    FwdArgs a;
    a.f = f;
    a.f_pitch = fp;
    a.out = out;
    a.out_pitch = op;
    a.H = p->H;
    a.W = p->W;
    a.R = p->R;
    a.taps = p->d_taps;
    a.hdr = p->d_hdr;
    a.pairs = p->d_pairs;
    a.cap_pairs = p->cap_pairs;
    a.set_tile = p->opt.t_mode == BF_T_TILE ? p->set_tile : 0;
    a.sets_x = p->sets_x;
    a.c0 = 0.5f * p->opt.value_range;
    a.n_guarded = p->d_nguard;
    a.den_out = nullptr;
    a.den_pitch = 0;
    a.h_taps = p->h_taps;
    a.sep_P = p->d_sep_P;
    a.sep_nd = p->d_sep_nd;
    a.sep_nk = p->sep_nk;
    a.sep_Wp = p->sep_Wp;
    a.sep_cap_terms = p->cap_pairs + 1;
    a.stall_test = p->stall_test;
    a.box_rs = box_running_sums(p->opt, p->R);
    a.box = p->opt.spatial == BF_SPATIAL_BOX;
    if (p->d_fix) {
        a.fix_list = p->d_fix;
        a.fix_count = p->d_fixcnt;
        a.fix_cap = p->fix_cap;
        a.fix_kappa = p->opt.plane_dtype == BF_PLANES_FP32 ? p->opt.fp32_recheck
                                                           : p->opt.lowp_recheck;
    }
    return a;
}

// The FP32 recheck of what a 16-bit forward with these arguments listed.
FixArgs fixup_args(bf_plan_s* p, const FwdArgs& fa)
{
    FixArgs x;
    x.f = fa.f;
    x.f_pitch = fa.f_pitch;
    x.out = fa.out;
    x.out_pitch = fa.out_pitch;
    x.H = p->H;
    x.W = p->W;
    x.R = p->R;
    x.taps = p->d_taps;
    x.hdr = p->d_hdr;
    x.pairs = p->d_pairs;
    x.cap_pairs = p->cap_pairs;
    x.set_tile = fa.set_tile;
    x.sets_x = p->sets_x;
    x.sigma_r = p->sigma_r;
    x.list = fa.fix_list;
    x.count = fa.fix_count;
    x.fix_cap = fa.fix_cap;
    x.n_guarded = p->d_nguard;
    x.set0 = 0;
    x.ntab = fixup_table_entries(p->n_cap);
    x.scan = p->d_fixscan;
    return x;
}

// Event k (0..3) of the current timed execute, or null when not timing.
static cudaEvent_t timing_event(bf_plan_s* p, int k)
{
    if (!p->timing || p->n_timed >= kMaxTimed) return nullptr;
    return p->ev[kEvPerExec * p->n_timed + k];
}

static cudaError_t mark(bf_plan_s* p, int k, cudaStream_t s)
{
    cudaEvent_t e = timing_event(p, k);
    return e ? cudaEventRecord(e, s) : cudaSuccess;
}

// Steps 1-5 of Algorithm 2 (T, N, M, pair table) on the plan's device.
cudaError_t enqueue_params(bf_plan_s* p, const float* f, size_t fp, cudaStream_t s)
{
    cudaError_t e = mark(p, 0, s);
    if (e != cudaSuccess) return e;
    if (p->opt.t_mode == BF_T_TILE && tile_params_ok(p->R, p->set_tile, p->n_cap)) {
        // T and the parameter set of every T-tile in one launch
        e = cudaMemsetAsync(p->d_nguard, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
        if (p->d_fixcnt) {
            e = cudaMemsetAsync(p->d_fixcnt, 0, sizeof(unsigned) * p->n_fixcnt, s);
            if (e != cudaSuccess) return e;
        }
        e = launch_tile_params(f, fp, p->H, p->W, p->R, p->set_tile, p->sets_x, 0, p->n_sets,
                               p->d_T, params_args(p), s);
        if (e != cudaSuccess) return e;
        e = mark(p, 1, s);
        if (e != cudaSuccess) return e;
        return mark(p, 2, s);
    }
    if (p->opt.t_mode != BF_T_FIXED) {
        e = cudaMemsetAsync(p->d_T, 0, sizeof(unsigned) * p->n_sets, s);
        if (e != cudaSuccess) return e;
        e = launch_local_range(f, fp, p->H, p->W, p->R,
                               p->opt.t_mode == BF_T_TILE ? p->set_tile : 0, p->sets_x, p->d_T, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(p->d_nguard, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (p->d_fixcnt) {
        e = cudaMemsetAsync(p->d_fixcnt, 0, sizeof(unsigned) * p->n_fixcnt, s);
        if (e != cudaSuccess) return e;
    }
    e = mark(p, 1, s);
    if (e != cudaSuccess) return e;
    e = launch_params(params_args(p), s);
    if (e != cudaSuccess) return e;
    return mark(p, 2, s);
}

// The raised-polynomial path: the range of each set's region (unless T is
// fixed), N and the Chebyshev nodes, then the fused tile kernel.
cudaError_t enqueue_poly(bf_plan_s* p, const float* f, size_t fp, float* out, size_t op,
                         cudaStream_t s)
{
    cudaError_t e = mark(p, 0, s);
    if (e != cudaSuccess) return e;
    const bool fixed = p->opt.t_mode == BF_T_FIXED;
    const int set_tile = p->opt.t_mode == BF_T_TILE ? p->set_tile : 0;
    if (!fixed) {
        e = launch_poly_range(f, fp, p->H, p->W, p->R, set_tile, p->sets_x, p->n_sets, p->d_mm, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(p->d_nguard, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    e = mark(p, 1, s);
    if (e != cudaSuccess) return e;
    PolyParamsArgs pa;
    pa.mm = fixed ? nullptr : p->d_mm;
    pa.n_sets = p->n_sets;
    pa.sigma_r = p->sigma_r;
    pa.t_fixed = p->opt.t_fixed;
    pa.value_range = p->opt.value_range;
    pa.n_cap = p->n_cap;
    pa.cap_nodes = p->cap_pairs;
    pa.hdr = p->d_hdr;
    pa.nodes = p->d_pairs;
    pa.status = p->d_status;
    e = launch_poly_params(pa, s);
    if (e != cudaSuccess) return e;
    e = mark(p, 2, s);
    if (e != cudaSuccess) return e;
    e = launch_poly32(forward_args(p, f, fp, out, op), s);
    if (e != cudaSuccess) return e;
    e = mark(p, 3, s);
    if (e != cudaSuccess) return e;
    return mark(p, 4, s);
}

// ---- host-to-host execution in row bands ---------------------------------
//
// With exact T per T-tile every quantity of a band of output rows depends on
// the input rows within R of it only: the T-tiles of the band (K1: windows of
// R around each pixel), their parameter sets (K2) and the band's output tiles
// (K3).  So the image is copied in (in chunks of one T-tile row, each with an
// event), filtered and copied out in bands of kHostBandRows rows, half that
// for the first and the last band so that the pipeline fills and drains
// sooner: band b is filtered once the chunk holding its last halo row is on
// the device, while later chunks are copied in and earlier bands out.  Two
// compute streams alternate so that one band's last wave of tiles overlaps
// the next band's first.  A band's FP32 recheck (16-bit planes) runs on a
// fifth stream of the lowest priority, the compute streams at the highest:
// pending forward tiles take the SMs first and the rechecks fill the gaps;
// a band is copied out after its recheck.  Same kernels, same arithmetic
// per pixel as bf_execute.  (4096^2, tuned: 1024-row bands 2.49 ms per call,
// 768 2.51, 512 2.54; with the rechecks on the compute streams 2.71 at 512.)
constexpr int kHostBandRows = 1024;
constexpr long long kMinSpinLimit = 1ll << 16;   // polls; see bf_plan

int host_band_rows(const bf_plan_s* p)
{
    const int t = p->set_tile > 0 ? p->set_tile : 128;
    return (std::max(kHostBandRows, t) + t - 1) / t * t;
}

bool host_banded(const bf_plan_s* p)
{
    int th = 0, tw = 0;
    fwd_tc_tile(&th, &tw);
    return p->opt.filter != BF_FILTER_YVV && p->opt.plane_dtype != BF_PLANES_FP32 &&
           p->opt.t_mode == BF_T_TILE && p->set_tile % th == 0 && p->R < p->set_tile &&
           p->H >= 2 * host_band_rows(p);
}

bf_status execute_host_banded(bf_plan_s* p, const float* fh, float* oh, cudaStream_t s)
{
    const int H = p->H, W = p->W, B = host_band_rows(p), C = p->set_tile;
    int th = 0, tw = 0;
    fwd_tc_tile(&th, &tw);
    // band boundaries (multiples of the T-tile): a half band first, full
    // bands, then what is left (at most a full band) last
    std::vector<int> cut{0};
    const int half = std::max(C, B / 2 / C * C);
    cut.push_back(std::min(H, half));
    while (cut.back() < H) cut.push_back(std::min(H, cut.back() + B));
    if (cut.size() > 3 && H - cut[cut.size() - 2] > half) {
        // split the last full band so that the last band is a half band too
        const int last0 = cut[cut.size() - 2];
        cut.back() = std::min(H, last0 + (H - last0 - half + C - 1) / C * C);
        if (cut.back() < H) cut.push_back(H);
    }
    const int nb = (int)cut.size() - 1;
    const int nc = (H + C - 1) / C;                  // copy chunks of one T-tile row
    const int need = 3 + nc + 2 * nb;
    if (!p->hst[0]) {
        // the compute streams at the highest priority, the recheck stream at
        // the lowest: pending forward tiles take the SMs first, and the
        // rechecks run in the gaps (a band's last partial wave)
        int least = 0, greatest = 0;
        BF_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        for (int i = 0; i < 5; ++i) {
            const int prio = (i == 1 || i == 2) ? greatest : (i == 4 ? least : 0);
            BF_CUDA(cudaStreamCreateWithPriority(&p->hst[i], cudaStreamNonBlocking, prio));
        }
    }
    if (p->n_hev < need) {
        if (p->hev) {
            for (int i = 0; i < p->n_hev; ++i)
                if (p->hev[i]) cudaEventDestroy(p->hev[i]);
            free(p->hev);
        }
        p->hev = (cudaEvent_t*)calloc(need, sizeof(cudaEvent_t));
        p->n_hev = 0;
        if (!p->hev) return BF_ERR_ALLOC;
        for (int i = 0; i < need; ++i)
            BF_CUDA(cudaEventCreateWithFlags(&p->hev[i], cudaEventDisableTiming));
        p->n_hev = need;
    }
    cudaEvent_t ev_fork = p->hev[0], ev_clear = p->hev[1], ev_join = p->hev[2];
    cudaEvent_t* ev_in = p->hev + 3;                 // per chunk
    cudaEvent_t* ev_done = p->hev + 3 + nc;          // per band
    cudaEvent_t* ev_fwd = p->hev + 3 + nc + nb;      // per band: forward done
    cudaStream_t s_in = p->hst[0], s_out = p->hst[3], s_fix = p->hst[4];
    BF_CUDA(cudaEventRecord(ev_fork, s));
    for (int i = 0; i < 5; ++i) BF_CUDA(cudaStreamWaitEvent(p->hst[i], ev_fork, 0));
    // T words and the guard counter start at zero for every band's kernels
    BF_CUDA(cudaMemsetAsync(p->d_T, 0, sizeof(unsigned) * p->n_sets, p->hst[1]));
    BF_CUDA(cudaMemsetAsync(p->d_nguard, 0, sizeof(unsigned long long), p->hst[1]));
    if (p->d_fixcnt)
        BF_CUDA(cudaMemsetAsync(p->d_fixcnt, 0, sizeof(unsigned) * p->n_fixcnt, p->hst[1]));
    BF_CUDA(cudaEventRecord(ev_clear, p->hst[1]));
    BF_CUDA(cudaStreamWaitEvent(p->hst[2], ev_clear, 0));
    const size_t row_bytes = sizeof(float) * (size_t)W;
    int copied = 0;                                  // chunks enqueued so far
    for (int b = 0; b < nb; ++b) {
        const int r0 = cut[b], r1 = cut[b + 1];
        // chunks up to the one holding input row r1 - 1 + R
        const int last_chunk = std::min(nc - 1, (std::min(H - 1, r1 - 1 + p->R)) / C);
        for (; copied <= last_chunk; ++copied) {
            const size_t c0 = (size_t)copied * C, rows = std::min(H - (int)c0, C);
            BF_CUDA(cudaMemcpyAsync(p->d_hin + c0 * W, fh + c0 * W, rows * row_bytes,
                                    cudaMemcpyHostToDevice, s_in));
            BF_CUDA(cudaEventRecord(ev_in[copied], s_in));
        }
        cudaStream_t cs = p->hst[1 + (b & 1)];
        const int rows = r1 - r0;
        BF_CUDA(cudaStreamWaitEvent(cs, ev_in[last_chunk], 0));
        const int bset0 = r0 / C * p->sets_x, bsets = (rows + C - 1) / C * p->sets_x;
        if (tile_params_ok(p->R, p->set_tile, p->n_cap)) {
            BF_CUDA(launch_tile_params(p->d_hin, W, H, W, p->R, p->set_tile, p->sets_x, bset0,
                                       bsets, p->d_T, params_args(p), cs));
        } else {
            BF_CUDA(launch_local_range(p->d_hin, W, H, W, p->R, p->set_tile, p->sets_x, p->d_T,
                                       cs, r0 / range_tile(),
                                       (rows + range_tile() - 1) / range_tile()));
            ParamsArgs pa = params_args(p);
            pa.set0 = bset0;
            BF_CUDA(launch_params(pa, cs, bsets));
        }
        FwdArgs fa = forward_args(p, p->d_hin, W, p->d_hout, W);
        fa.y_tile0 = r0 / th;
        fa.y_tiles = (rows + th - 1) / th;
        BF_CUDA(launch_fwd_tc(fa, p->opt.plane_dtype == BF_PLANES_BF16, p->opt.spin_limit,
                              p->d_status, cs));
        if (p->d_fix) {                          // the band's own sets, on the recheck stream
            BF_CUDA(cudaEventRecord(ev_fwd[b], cs));
            BF_CUDA(cudaStreamWaitEvent(s_fix, ev_fwd[b], 0));
            FixArgs xa = fixup_args(p, fa);
            xa.set0 = r0 / C * p->sets_x;
            xa.scan = p->d_fixscan + xa.set0 + b;    // own offsets per band
            BF_CUDA(launch_fixup(xa, (rows + C - 1) / C * p->sets_x, s_fix));
            BF_CUDA(cudaEventRecord(ev_done[b], s_fix));
        } else {
            BF_CUDA(cudaEventRecord(ev_done[b], cs));
        }
        BF_CUDA(cudaStreamWaitEvent(s_out, ev_done[b], 0));
        BF_CUDA(cudaMemcpyAsync(oh + (size_t)r0 * W, p->d_hout + (size_t)r0 * W,
                                (size_t)rows * row_bytes, cudaMemcpyDeviceToHost, s_out));
    }
    // join every side stream into the caller's stream
    BF_CUDA(cudaEventRecord(ev_join, s_out));
    BF_CUDA(cudaStreamWaitEvent(s, ev_join, 0));
    BF_CUDA(cudaEventRecord(ev_clear, p->hst[2]));
    BF_CUDA(cudaStreamWaitEvent(s, ev_clear, 0));
    BF_CUDA(cudaEventRecord(ev_fork, s_in));
    BF_CUDA(cudaStreamWaitEvent(s, ev_fork, 0));
    BF_CUDA(cudaStreamSynchronize(s));
    p->executed = 1;
    p->last = s;
    return BF_OK;
}

}  // namespace bf

extern "C" {

void bf_options_init(bf_options* o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->t_mode = BF_T_GLOBAL;
    o->t_fixed = 0.f;
    o->value_range = 255.f;
    o->trunc_rule = BF_RULE_ALG2;
    o->filter = BF_FILTER_AUTO;
    o->plane_dtype = BF_PLANES_FP32;
    o->n_max = 4096;
    o->t_tile = 64;
    o->spin_limit = 1ll << 22;
    o->spatial = BF_SPATIAL_GAUSS;
    o->lowp_recheck = 0.05f;
    o->fp32_recheck = 0.05f;
}

const char* bf_status_string(bf_status s)
{
    switch (s) {
    case BF_OK: return "ok";
    case BF_ERR_INVALID_ARG: return "invalid argument";
    case BF_ERR_ORDER_TOO_LARGE: return "order N above the plan's cap";
    case BF_ERR_ALLOC: return "allocation failed";
    case BF_ERR_CUDA: return "CUDA runtime error";
    case BF_ERR_TIMEOUT: return "bounded device wait ran out";
    case BF_ERR_NO_FORWARD: return "backward before any forward";
    case BF_ERR_NOT_SUPPORTED: return "option combination not supported";
    case BF_ERR_DEVICE_STATUS: return "device status word holds an error";
    }
    return "unknown status";
}

bf_status bf_plan(int H, int W, double sigma_s, double sigma_r, double eps, const bf_options* opt,
                  bf_plan_t* out)
{
    if (!out) return BF_ERR_INVALID_ARG;
    *out = nullptr;
    bf_options o;
    if (opt) o = *opt;
    else bf_options_init(&o);
    if (H < 1 || W < 1 || H > (1 << 16) || W > (1 << 16)) return BF_ERR_INVALID_ARG;
    if (!(sigma_s > 0.0) || !(sigma_r > 0.0) || !(eps >= 0.0) || !(eps < 1.0))
        return BF_ERR_INVALID_ARG;
    if (!isfinite(sigma_s) || !isfinite(sigma_r)) return BF_ERR_INVALID_ARG;
    if (o.t_mode < BF_T_FIXED || o.t_mode > BF_T_TILE) return BF_ERR_INVALID_ARG;
    if (o.trunc_rule < BF_RULE_ALG2 || o.trunc_rule > BF_RULE_CHERNOFF) return BF_ERR_INVALID_ARG;
    if (!(o.value_range > 0.f) || !isfinite(o.value_range)) return BF_ERR_INVALID_ARG;
    if (o.n_max < 1) return BF_ERR_INVALID_ARG;
    if (!(o.lowp_recheck >= 0.f) || !(o.lowp_recheck < 1.f)) return BF_ERR_INVALID_ARG;
    if (!(o.fp32_recheck >= 0.f) || !(o.fp32_recheck < 1.f)) return BF_ERR_INVALID_ARG;
    if (o.n_max > 4096) return BF_ERR_NOT_SUPPORTED;
    for (int i = 0; i < (int)(sizeof(o.reserved) / sizeof(o.reserved[0])); ++i)
        if (o.reserved[i]) return BF_ERR_INVALID_ARG;
    // the box filter (Sec. 4): sigma_s is its radius, a whole number of pixels
    const bool box = o.spatial == BF_SPATIAL_BOX;
    if (o.spatial != BF_SPATIAL_GAUSS && !box) return BF_ERR_INVALID_ARG;
    if (box && (sigma_s < 1.0 || sigma_s != floor(sigma_s))) return BF_ERR_INVALID_ARG;
    if (box && o.filter == BF_FILTER_YVV) return BF_ERR_NOT_SUPPORTED;
    if (o.filter == BF_FILTER_AUTO) o.filter = BF_FILTER_FIR;
    if (o.filter != BF_FILTER_FIR && o.filter != BF_FILTER_YVV) return BF_ERR_INVALID_ARG;
    if (o.plane_dtype < BF_PLANES_FP32 || o.plane_dtype > BF_PLANES_FP16) return BF_ERR_INVALID_ARG;
    const bool poly = o.range_kernel == BF_RANGE_POLY;
    if (o.range_kernel != BF_RANGE_COSINE && !poly) return BF_ERR_INVALID_ARG;
    if (poly && (o.filter != BF_FILTER_FIR || o.plane_dtype != BF_PLANES_FP32))
        return BF_ERR_NOT_SUPPORTED;
    // non-local means: a 3 x 3 patch mask holding the centre
    const bool nlm = o.patch_mask != 0;
    if (nlm && (o.patch_mask < 0 || o.patch_mask >= (1 << 9) || !(o.patch_mask & (1 << 4))))
        return BF_ERR_INVALID_ARG;
    if (nlm && (poly || o.filter == BF_FILTER_YVV || o.plane_dtype != BF_PLANES_FP32 ||
                o.t_mode == BF_T_TILE))
        return BF_ERR_NOT_SUPPORTED;
    // the recursive filter: FP32 planes, one parameter set per image (every
    // output depends on the whole image), and the recursion's range of scales
    YvvCoef yc;
    if (o.filter == BF_FILTER_YVV &&
        (o.plane_dtype != BF_PLANES_FP32 || o.t_mode == BF_T_TILE || !yvv_design(sigma_s, &yc, nullptr)))
        return BF_ERR_NOT_SUPPORTED;
    if (o.t_mode == BF_T_TILE && (o.t_tile < 64 || o.t_tile % 64)) return BF_ERR_INVALID_ARG;
    // the 16-bit planes run on the tensor cores with 128 x 32 output tiles,
    // which must nest inside the T-tiles
    if (o.plane_dtype != BF_PLANES_FP32 && o.t_mode == BF_T_TILE && o.t_tile % 128)
        return BF_ERR_INVALID_ARG;
    if (o.t_mode == BF_T_FIXED && !(o.t_fixed > 0.f)) o.t_fixed = o.value_range;
    // the polynomial expansion spans [0, value_range] with a fixed T
    if (poly && o.t_mode == BF_T_FIXED && o.t_fixed < o.value_range) return BF_ERR_NOT_SUPPORTED;
    if (o.spin_limit <= 0) o.spin_limit = 1ll << 22;
    // the same bound limits the wait that lets issued MMAs finish before a
    // stopping CTA frees its TMEM: keep it far above their completion time
    if (o.spin_limit < kMinSpinLimit) o.spin_limit = kMinSpinLimit;   // floor for normal runs

    const double Rr = box ? sigma_s : ceil(3.0 * sigma_s);
    if (Rr > 1000.0) return BF_ERR_NOT_SUPPORTED;
    const int R = (int)Rr;
    if (!poly && o.t_mode != BF_T_FIXED && R > range_max_radius()) return BF_ERR_NOT_SUPPORTED;
    int th = 0, tw = 0;
    const bool box_rs = box_running_sums(o, R);
    const bool use_sep = !poly && !box_rs && o.filter == BF_FILTER_FIR &&
                         o.plane_dtype == BF_PLANES_FP32 && o.t_mode != BF_T_TILE &&
                         !fwd32t_ok(R, 0) && sep32_ok(R);
    const double Tcap = o.t_mode == BF_T_FIXED ? (double)o.t_fixed : (double)o.value_range;
    int n_cap = poly ? poly_order_of(Tcap, sigma_r) : order_of(Tcap, sigma_r);
    if (o.t_mode == BF_T_FIXED && n_cap > o.n_max) return BF_ERR_ORDER_TOO_LARGE;
    if (n_cap > o.n_max) n_cap = o.n_max;
    if (poly) {
        poly_tile(R, 2 * n_cap + 1, &th, &tw);
        if (o.t_mode == BF_T_TILE && th > 0 && o.t_tile % th) th = tw = 0;
    } else if (nlm) {
        int p = 0;
        for (int b = 0; b < 9; ++b) p += (o.patch_mask >> b) & 1;
        double terms = 1.0;
        for (int i = 0; i < p; ++i) terms *= (double)(n_cap + 1);
        if (terms > (double)(1 << 22)) return BF_ERR_NOT_SUPPORTED;
        nlm_tile(R, n_cap, &th, &tw);
    } else if (o.filter == BF_FILTER_YVV) {
        th = tw = 1;                      // whole lines, no output tiles
    } else if (use_sep) {
        th = 128;                         // column-pass tile of the two-pass FIR
        tw = 32;
    } else if (o.plane_dtype == BF_PLANES_FP32 && box_rs) {
        th = box32_rows(R, o.t_mode == BF_T_TILE ? o.t_tile : 0);
        tw = 32;
    } else if (o.plane_dtype == BF_PLANES_FP32) {
        fwd32_tile(R, &th, &tw);
        const int st = o.t_mode == BF_T_TILE ? o.t_tile : 0;
        if (fwd32t_ok(R, st)) {
            th = fwd32t_rows(st);
            tw = 32;
        }
    } else if (R <= fwd_tc_max_radius()) {
        fwd_tc_tile(&th, &tw);
    }
    if (!th) return BF_ERR_NOT_SUPPORTED;

    bf_plan_s* p = (bf_plan_s*)calloc(1, sizeof(bf_plan_s));
    if (!p) return BF_ERR_ALLOC;
    p->H = H;
    p->W = W;
    p->R = R;
    p->sigma_s = sigma_s;
    p->sigma_r = sigma_r;
    p->eps = eps;
    p->opt = o;
    p->th = th;
    p->tw = tw;
    p->c0 = 0.5f * o.value_range;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        free(p);
        return BF_ERR_CUDA;
    }
    if (o.t_mode == BF_T_TILE) {
        p->set_tile = o.t_tile;
        p->sets_x = (W + o.t_tile - 1) / o.t_tile;
        p->sets_y = (H + o.t_tile - 1) / o.t_tile;
    } else {
        p->set_tile = 0;
        p->sets_x = p->sets_y = 1;
    }
    p->n_sets = p->sets_x * p->sets_y;
    p->n_cap = n_cap;
    p->cap_pairs = poly ? 2 * n_cap + 1 : n_cap / 2 + 1;   // pairs, or the polynomial's nodes
    if (nlm) {                          // patch pixels, the centre first
        p->patch_uy[0] = p->patch_ux[0] = 0;
        p->patch_p = 1;
        for (int b = 0; b < 9; ++b)
            if (b != 4 && ((o.patch_mask >> b) & 1)) {
                p->patch_uy[p->patch_p] = b / 3 - 1;
                p->patch_ux[p->patch_p] = b % 3 - 1;
                ++p->patch_p;
            }
    }

    bool ok = true;
    ok &= cudaMalloc(&p->d_T, sizeof(unsigned) * p->n_sets) == cudaSuccess;
    ok &= cudaMalloc(&p->d_hdr, sizeof(SetHdr) * p->n_sets) == cudaSuccess;
    ok &= cudaMalloc(&p->d_pairs, sizeof(Pair) * (size_t)p->n_sets * p->cap_pairs) == cudaSuccess;
    ok &= cudaMalloc(&p->d_taps, sizeof(float) * (2 * R + 1)) == cudaSuccess;
    ok &= cudaMalloc(&p->d_logfact, sizeof(double) * (n_cap + 1)) == cudaSuccess;
    ok &= cudaMalloc(&p->d_status, sizeof(unsigned)) == cudaSuccess;
    ok &= cudaMalloc(&p->d_nguard, sizeof(unsigned long long)) == cudaSuccess;
    if (poly) ok &= cudaMalloc(&p->d_mm, sizeof(unsigned) * 2 * p->n_sets) == cudaSuccess;
    if (!ok) {
        free_plan(p);
        return BF_ERR_ALLOC;
    }
    // spatial taps g(k) = exp(-k^2 / (2 sigma_s^2)) (1 for the box) and the
    // log(k!) table
    float* taps = (float*)malloc(sizeof(float) * (2 * R + 1));
    double* lf = (double*)malloc(sizeof(double) * (n_cap + 1));
    if (!taps || !lf) {
        free(taps);
        free(lf);
        free_plan(p);
        return BF_ERR_ALLOC;
    }
    for (int k = -R; k <= R; ++k)
        taps[k + R] = box ? 1.f : (float)exp(-(double)k * (double)k / (2.0 * sigma_s * sigma_s));
    for (int k = 0; k <= n_cap; ++k) lf[k] = lgamma((double)k + 1.0);
    ok &= cudaMemcpy(p->d_taps, taps, sizeof(float) * (2 * R + 1), cudaMemcpyHostToDevice) ==
          cudaSuccess;
    ok &= cudaMemcpy(p->d_logfact, lf, sizeof(double) * (n_cap + 1), cudaMemcpyHostToDevice) ==
          cudaSuccess;
    ok &= cudaMemset(p->d_status, 0, sizeof(unsigned)) == cudaSuccess;
    ok &= cudaMemset(p->d_nguard, 0, sizeof(unsigned long long)) == cudaSuccess;
    p->h_taps = taps;      // kept: the tall FP32 kernel takes the taps as a parameter
    free(lf);
    if (o.t_mode == BF_T_FIXED) {
        float T = o.t_fixed;
        ok &= cudaMemcpy(p->d_T, &T, sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    // FP32 planes take the recheck where the window is large (R > 24: the
    // two-pass FIR, the small FIR tiles, the box's running sums) and the
    // recheck kernel's window fits (R <= 63); the FIR of the cosine kernel
    // only (not the recursive filter, the polynomial or the patch kernels)
    const bool fp32_fix = o.plane_dtype == BF_PLANES_FP32 && o.fp32_recheck > 0.f && R > 24 &&
                          R <= 63 && o.filter == BF_FILTER_FIR && !poly && !nlm;
    if (ok && ((o.plane_dtype != BF_PLANES_FP32 && o.lowp_recheck > 0.f) || fp32_fix)) {
        // the recheck lists (a slot per pixel of each set's region, so they
        // cannot overflow) and one list length per set
        p->n_fixcnt = p->n_sets;
        p->fix_cap = o.t_mode == BF_T_TILE ? (unsigned)(o.t_tile * o.t_tile) : (unsigned)H * W;
        if (cudaMalloc(&p->d_fix, sizeof(unsigned) * (size_t)p->n_sets * p->fix_cap) != cudaSuccess ||
            cudaMalloc(&p->d_fixcnt, sizeof(unsigned) * p->n_fixcnt) != cudaSuccess ||
            cudaMalloc(&p->d_fixscan, sizeof(unsigned) * (p->n_sets + H / 64 + 8)) != cudaSuccess) {
            cudaGetLastError();
            free_plan(p);
            return BF_ERR_ALLOC;
        }
        ok &= cudaMemset(p->d_fixcnt, 0, sizeof(unsigned) * p->n_fixcnt) == cudaSuccess;
    }
    if (ok && use_sep) {
        // row-filtered planes of sep_nk terms at a time (up to 2 GiB), and
        // the (num, den) partial carried between chunks of terms
        p->sep_Wp = sep32_width(W);
        const size_t per_term = (size_t)4 * H * p->sep_Wp * sizeof(float);
        const size_t budget = (size_t)2 << 30;
        const int cap_terms = p->cap_pairs + 1;
        size_t nk = budget / per_term;
        if (nk < 1) nk = 1;
        if (nk > (size_t)cap_terms) nk = cap_terms;
        p->sep_nk = (int)nk;
        if (cudaMalloc(&p->d_sep_P, nk * per_term) != cudaSuccess ||
            cudaMalloc(&p->d_sep_nd, (size_t)H * W * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            free_plan(p);
            return BF_ERR_ALLOC;
        }
    }
    if (ok && o.filter == BF_FILTER_YVV) {
        // terms per pass from the cap (pairs + zero frequency); workspace:
        // row-filtered planes [H][W][C] x 16 B, (num, den) [H][W], masses
        const int cap_terms = p->cap_pairs + 1;
        p->yvv_C = yvv_terms_per_pass(cap_terms);
        p->yvv_G = 32 / p->yvv_C;
        p->yvv_passes = (cap_terms + p->yvv_C - 1) / p->yvv_C;
        const size_t npx = (size_t)H * W;
        const size_t nst = (size_t)H * ((W + 7) / 8) * 3 * 32;
        if (cudaMalloc(&p->d_yvv_P, npx * 32 * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&p->d_yvv_S, nst * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&p->d_yvv_nd, npx * p->yvv_G * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&p->d_yvv_mass, sizeof(float) * ((size_t)H + W)) != cudaSuccess) {
            cudaGetLastError();
            free_plan(p);
            return BF_ERR_ALLOC;
        }
        float* m = (float*)malloc(sizeof(float) * ((size_t)H + W));
        if (!m) {
            free_plan(p);
            return BF_ERR_ALLOC;
        }
        yvv_line_mass(sigma_s, H, m);
        yvv_line_mass(sigma_s, W, m + H);
        ok &= cudaMemcpy(p->d_yvv_mass, m, sizeof(float) * ((size_t)H + W),
                         cudaMemcpyHostToDevice) == cudaSuccess;
        free(m);
    }
    if (!ok) {
        free_plan(p);
        return BF_ERR_CUDA;
    }
    *out = p;
    return BF_OK;
}

bf_status bf_execute(bf_plan_t p, const float* f, size_t fp, float* out, size_t op, void* stream)
{
    if (!p || !f || !out) return BF_ERR_INVALID_ARG;
    if (fp < (size_t)p->W || op < (size_t)p->W) return BF_ERR_INVALID_ARG;
    if ((const void*)f == (const void*)out) return BF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    BF_CUDA(cudaSetDevice(p->device));
    if (p->opt.range_kernel == BF_RANGE_POLY) {
        BF_CUDA(enqueue_poly(p, f, fp, out, op, s));
        if (p->timing && p->n_timed < kMaxTimed) ++p->n_timed;
        p->executed = 1;
        p->last = s;
        return BF_OK;
    }
    BF_CUDA(enqueue_params(p, f, fp, s));
    if (p->patch_p) {
        NlmPatch pt;
        pt.p = p->patch_p;
        for (int i = 0; i < 9; ++i) {
            pt.uy[i] = p->patch_uy[i];
            pt.ux[i] = p->patch_ux[i];
        }
        pt.sigma_r = (float)p->sigma_r;
        BF_CUDA(launch_nlm32(forward_args(p, f, fp, out, op), pt, p->n_cap, s));
    } else if (p->opt.filter == BF_FILTER_YVV)
        BF_CUDA(launch_yvv(yvv_args(p, f, fp, out, op), p->yvv_C, p->yvv_passes, s));
    else if (p->opt.plane_dtype == BF_PLANES_FP32)
        BF_CUDA(launch_fwd32(forward_args(p, f, fp, out, op), s));
    else
        BF_CUDA(launch_fwd_tc(forward_args(p, f, fp, out, op),
                              p->opt.plane_dtype == BF_PLANES_BF16, p->opt.spin_limit,
                              p->d_status, s));
    BF_CUDA(mark(p, 3, s));
    if (p->d_fix)          // 16-bit planes, or FP32 planes with R > 24: the FP32 recheck
        BF_CUDA(launch_fixup(fixup_args(p, forward_args(p, f, fp, out, op)), p->n_sets, s));
    BF_CUDA(mark(p, 4, s));
    if (p->timing && p->n_timed < kMaxTimed) ++p->n_timed;
    p->executed = 1;
    p->last = s;
    return BF_OK;
}

bf_status bf_execute_host(bf_plan_t p, const float* fh, float* oh, void* stream)
{
    if (!p || !fh || !oh) return BF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    BF_CUDA(cudaSetDevice(p->device));
    const size_t bytes = sizeof(float) * (size_t)p->H * p->W;
    if (!p->d_hin) {
        if (cudaMalloc(&p->d_hin, bytes) != cudaSuccess) return BF_ERR_ALLOC;
        if (cudaMalloc(&p->d_hout, bytes) != cudaSuccess) return BF_ERR_ALLOC;
    }
    if (host_banded(p)) return execute_host_banded(p, fh, oh, s);
    BF_CUDA(cudaMemcpyAsync(p->d_hin, fh, bytes, cudaMemcpyHostToDevice, s));
    bf_status st = bf_execute(p, p->d_hin, p->W, p->d_hout, p->W, stream);
    if (st != BF_OK) return st;
    BF_CUDA(cudaMemcpyAsync(oh, p->d_hout, bytes, cudaMemcpyDeviceToHost, s));
    BF_CUDA(cudaStreamSynchronize(s));
    return BF_OK;
}

bf_status bf_backward(bf_plan_t p, const float* f, const float* gout, float* gin, size_t pitch,
                      void* stream)
{
    if (!p || !f || !gout || !gin) return BF_ERR_INVALID_ARG;
    if (pitch < (size_t)p->W) return BF_ERR_INVALID_ARG;
    if (p->opt.filter == BF_FILTER_YVV || p->opt.range_kernel == BF_RANGE_POLY || p->patch_p)
        return BF_ERR_NOT_SUPPORTED;
    if (!p->executed) return BF_ERR_NO_FORWARD;
    cudaStream_t s = (cudaStream_t)stream;
    BF_CUDA(cudaSetDevice(p->device));
    cudaError_t e = launch_backward(p, f, gout, gin, pitch, s);
    if (e == cudaErrorNotSupported) return BF_ERR_NOT_SUPPORTED;
    if (e == cudaErrorMemoryAllocation) return BF_ERR_ALLOC;
    BF_CUDA(e);
    p->last = s;
    return BF_OK;
}

bf_status bf_get_info(bf_plan_t p, bf_info* info)
{
    if (!p || !info) return BF_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    info->H = p->H;
    info->W = p->W;
    info->R = p->R;
    info->n_sets = p->n_sets;
    info->filter = p->opt.filter;
    info->plane_dtype = p->opt.plane_dtype;
    info->t_mode = p->opt.t_mode;
    info->tile_h = p->th;
    info->tile_w = p->tw;
    BF_CUDA(cudaSetDevice(p->device));
    BF_CUDA(cudaStreamSynchronize(p->last));
    if (!p->executed) return BF_OK;
    SetHdr* h = (SetHdr*)malloc(sizeof(SetHdr) * p->n_sets);
    if (!h) return BF_ERR_ALLOC;
    unsigned long long ng = 0;
    unsigned st = 0;
    std::vector<unsigned> fc(p->n_fixcnt);
    bool ok = cudaMemcpy(h, p->d_hdr, sizeof(SetHdr) * p->n_sets, cudaMemcpyDeviceToHost) ==
              cudaSuccess;
    ok &= cudaMemcpy(&ng, p->d_nguard, sizeof(ng), cudaMemcpyDeviceToHost) == cudaSuccess;
    ok &= cudaMemcpy(&st, p->d_status, sizeof(st), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (p->n_fixcnt)
        ok &= cudaMemcpy(fc.data(), p->d_fixcnt, sizeof(unsigned) * p->n_fixcnt,
                         cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) {
        free(h);
        return BF_ERR_CUDA;
    }
    for (unsigned v : fc) info->n_rechecked += v;
    int best = 0;
    long long terms = 0;
    float Tm = 0.f;
    for (int i = 0; i < p->n_sets; ++i) {
        if (h[i].N > h[best].N) best = i;
        if (h[i].T > Tm) Tm = h[i].T;
        if (h[i].F >= 0) terms += p->opt.range_kernel == BF_RANGE_POLY ? h[i].F
                                                                       : h[i].N - 2 * h[i].M + 1;
    }
    info->T = Tm;
    info->N = h[best].N;
    info->M = h[best].M;
    // terms: N - 2M + 1 cosines, or the polynomial's 2N + 1 basis functions
    info->K = p->opt.range_kernel == BF_RANGE_POLY ? 2 * h[best].N + 1
                                                   : h[best].N - 2 * h[best].M + 1;
    info->n_guarded = (long long)ng;
    info->terms_total = terms;
    info->device_status = st;
    free(h);
    return BF_OK;
}

bf_status bf_get_sets(bf_plan_t p, float* T, int* N, int* M, int n)
{
    if (!p || n != p->n_sets) return BF_ERR_INVALID_ARG;
    if (!p->executed) return BF_ERR_NO_FORWARD;
    BF_CUDA(cudaSetDevice(p->device));
    BF_CUDA(cudaStreamSynchronize(p->last));
    SetHdr* h = (SetHdr*)malloc(sizeof(SetHdr) * n);
    if (!h) return BF_ERR_ALLOC;
    if (cudaMemcpy(h, p->d_hdr, sizeof(SetHdr) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        free(h);
        return BF_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i) {
        if (T) T[i] = h[i].T;
        if (N) N[i] = h[i].N;
        if (M) M[i] = h[i].M;
    }
    free(h);
    return BF_OK;
}

bf_status bf_get_device_status(bf_plan_t p, unsigned* bits)
{
    if (!p) return BF_ERR_INVALID_ARG;
    BF_CUDA(cudaSetDevice(p->device));
    BF_CUDA(cudaStreamSynchronize(p->last));
    unsigned st = 0;
    BF_CUDA(cudaMemcpy(&st, p->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    BF_CUDA(cudaMemset(p->d_status, 0, sizeof(unsigned)));
    if (bits) *bits = st;
    return st ? BF_ERR_DEVICE_STATUS : BF_OK;
}

void bf_destroy(bf_plan_t p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    cudaStreamSynchronize(p->last);
    batch_forget(p);
    free_plan(p);
}

bf_status bf_set_timing(bf_plan_t p, int on)
{
    if (!p) return BF_ERR_INVALID_ARG;
    BF_CUDA(cudaSetDevice(p->device));
    if (on && !p->ev) {
        p->ev = (cudaEvent_t*)calloc(kEvPerExec * kMaxTimed, sizeof(cudaEvent_t));
        if (!p->ev) return BF_ERR_ALLOC;
        for (int i = 0; i < kEvPerExec * kMaxTimed; ++i) BF_CUDA(cudaEventCreate(&p->ev[i]));
    }
    p->timing = on ? 1 : 0;
    p->n_timed = 0;
    return BF_OK;
}

bf_status bf_get_timing(bf_plan_t p, double* ms, int* count)
{
    if (!p || !ms) return BF_ERR_INVALID_ARG;
    BF_CUDA(cudaSetDevice(p->device));
    BF_CUDA(cudaStreamSynchronize(p->last));
    ms[0] = ms[1] = ms[2] = ms[3] = 0.0;
    for (int i = 0; i < p->n_timed; ++i) {
        float t;
        for (int k = 0; k < kEvPerExec - 1; ++k) {
            BF_CUDA(cudaEventElapsedTime(&t, p->ev[kEvPerExec * i + k],
                                         p->ev[kEvPerExec * i + k + 1]));
            ms[k] += t;
        }
    }
    if (count) *count = p->n_timed;
    p->n_timed = 0;
    return BF_OK;
}

bf_status bf_test_stall(bf_plan_t p, int on)
{
    if (!p) return BF_ERR_INVALID_ARG;
    if (p->opt.plane_dtype == BF_PLANES_FP32 || p->opt.filter == BF_FILTER_YVV)
        return BF_ERR_NOT_SUPPORTED;
    p->stall_test = on ? 1 : 0;
    return BF_OK;
}

bf_status bf_maxmin(const float* f, int H, int W, size_t pitch, int R, float* Mx, float* mn,
                    void* stream)
{
    if (!f || !Mx || !mn || H < 1 || W < 1 || R < 0 || pitch < (size_t)W)
        return BF_ERR_INVALID_ARG;
    if (R > range_max_radius()) return BF_ERR_NOT_SUPPORTED;
    return cuda_status(launch_maxmin(f, pitch, H, W, R, Mx, mn, (cudaStream_t)stream));
}



}  // extern "C"

namespace bf {

// Backward: a forward pass with FP32 planes on the parameters the last
// bf_execute left on device (writing out and den to plan scratch), then the
// adjoint kernel.  The scratch (two H x W images and a counter) is allocated
// by the first backward of the plan.
cudaError_t launch_backward(bf_plan_s* p, const float* f, const float* gout, float* gin,
                            size_t pitch, cudaStream_t s)
{
    int th = 0, tw = 0;
    bwd32_tile(p->R, &th, &tw);
    if (!th) return cudaErrorNotSupported;
    const size_t hw = (size_t)p->H * p->W;
    if (!p->d_bwd) {
        cudaError_t e = cudaMalloc(&p->d_bwd, sizeof(float) * (2 * hw + 4));
        if (e != cudaSuccess) return cudaErrorMemoryAllocation;
    }
    float* s_out = p->d_bwd;
    float* s_den = p->d_bwd + hw;
    unsigned long long* s_cnt =
        reinterpret_cast<unsigned long long*>(p->d_bwd + 2 * hw + ((2 * hw) & 1));
    FwdArgs fa = forward_args(p, f, pitch, s_out, p->W);
    fa.den_out = s_den;
    fa.den_pitch = p->W;
    fa.n_guarded = s_cnt;
    fa.fix_list = nullptr;     // the adjoint's forward is the FP32-plane filter itself, no recheck
    fa.fix_count = nullptr;
    cudaError_t e = launch_fwd32(fa, s);
    if (e != cudaSuccess) return e;
    BwdArgs ba;
    ba.h_taps = p->h_taps;
    ba.f = f;
    ba.u = gout;
    ba.grad = gin;
    ba.pitch = pitch;
    ba.out = s_out;
    ba.den = s_den;
    ba.spitch = p->W;
    ba.H = p->H;
    ba.W = p->W;
    ba.R = p->R;
    ba.taps = p->d_taps;
    ba.hdr = p->d_hdr;
    ba.pairs = p->d_pairs;
    ba.cap_pairs = p->cap_pairs;
    ba.set_tile = fa.set_tile;
    ba.sets_x = p->sets_x;
    ba.c0 = fa.c0;
    return launch_bwd32(ba, s);
}

}  // namespace bf
