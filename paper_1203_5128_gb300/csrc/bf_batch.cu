// bf_execute_batch: Algorithm 2 on many images of uneven sizes, each with its
// own plan (sigma_s, sigma_r, eps), as one graph of four launches:
//
//   1. clear the T words, guard counters and queue heads of the batch;
//   2. K1 batched: CTAs stride over every (image, 64 x 64 block) item;
//   3. K2 batched: one block per parameter set of every image;
//   4. K4: one persistent launch per tile shape, CTAs taking (image, tile)
//      items from an atomic queue head, costliest first (longest-processing-
//      time order), each item run by the same tile body as bf_execute.
//
// Images whose radius is beyond the fused tall tile (and whose plan holds the
// two-pass workspace) run the two-pass FIR instead, images large enough to
// fill a quarter of the GPU with the fused tall tile run that kernel, and
// images with 16-bit planes run the tensor-core kernel and its FP32 recheck:
// all as their own launches, after the batched K1 and K2, on side streams of
// the capture that the graph runs concurrently with the queue.
//
// The FP32 forward's arithmetic per output does not depend on the tile shape
// (every FIR sums its nonzero taps in increasing order; zero-padded taps add
// exact zeros), so the batch output equals bf_execute's bit for bit whatever
// shape serves an image.  The shape for each radius R is picked by a small
// autotuner: the first time a batch holds an image with that R, every shape
// whose shared memory fits is timed (CUDA events) on that image's first
// tiles and the fastest is remembered for the process.
//
// The graph is captured once per (plans, images) combination and cached;
// bf_destroy drops the cached graphs that name the destroyed plan.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "bf_internal.cuh"

using namespace bf;

namespace bf {
cudaError_t enqueue_params(bf_plan_s* p, const float* f, size_t fp, cudaStream_t s);
}
cudaError_t launch_batch_clear(const void* zeros, int n_zeros, unsigned* heads, int n_heads,
                               cudaStream_t s);

namespace {

struct BatchState {
    std::vector<const void*> key;
    int device = 0;
    cudaGraphExec_t exec = nullptr;
    void* blob = nullptr;
};

std::mutex g_mu;
std::map<std::vector<const void*>, BatchState*> g_states;
std::map<int, std::pair<int, int>> g_tile_choice;   // R -> (th, tw), per process

void free_state(BatchState* st)
{
    if (!st) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(st->device);
    if (st->exec) cudaGraphExecDestroy(st->exec);
    cudaFree(st->blob);
    cudaSetDevice(cur);
    delete st;
}

// Bytes of a host vector, rounded up so that the next array stays 256-byte aligned.
template <class T>
size_t padded_bytes(const std::vector<T>& v)
{
    return (v.size() * sizeof(T) + 255) / 256 * 256;
}

// Times one launch of each candidate shape of the FP32 forward on image f of
// plan p (after K1 + K2 of that image) and returns the fastest.
std::pair<int, int> autotune_tile(bf_plan_s* p, const float* f, float* out, cudaStream_t s)
{
    static const int shapes[][2] = {{64, 32}, {32, 32}, {16, 16}};
    std::pair<int, int> best(0, 0);
    float best_ms = 1e30f;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return best;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return best;
    }
    if (enqueue_params(p, f, p->W, s) == cudaSuccess) {
        FwdArgs fa = forward_args(p, f, p->W, out, p->W);
        for (auto& sh : shapes) {
            if (fwd32_smem(p->R, sh[0], sh[1]) > 227 * 1024) continue;
            // the items of the image's first rows of tiles, through the persistent kernel
            std::vector<int4> items;
            for (int by = 0; by < p->H && (int)items.size() < 512; by += sh[0])
                for (int bx = 0; bx < p->W; bx += sh[1]) items.push_back(make_int4(0, by, bx, 0));
            // the descriptor and items live in a temporary device buffer
            const size_t nb = 256 + padded_bytes(items) + 256;
            void* buf = nullptr;
            if (cudaMalloc(&buf, nb) != cudaSuccess) continue;
            char* c = static_cast<char*>(buf);
            FwdArgs* dA = reinterpret_cast<FwdArgs*>(c);
            int4* dI = reinterpret_cast<int4*>(c + 256);
            unsigned* dH = reinterpret_cast<unsigned*>(c + 256 + padded_bytes(items));
            cudaMemcpy(dA, &fa, sizeof(fa), cudaMemcpyHostToDevice);
            cudaMemcpy(dI, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
            const int per = fwd32_persistent_ctas_per_sm(sh[0], sh[1], p->R);
            float ms = 1e30f;
            if (per > 0) {
                for (int rep = 0; rep < 2; ++rep) {      // first run warms up
                    cudaMemsetAsync(dH, 0, sizeof(unsigned), s);
                    cudaEventRecord(a, s);
                    launch_fwd32_persistent(sh[0], sh[1], p->R, dA, dI, (int)items.size(), dH,
                                            sms * per, s);
                    cudaEventRecord(b, s);
                }
                if (cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
                ms /= (float)items.size();               // per tile of this shape ...
                ms /= (float)(sh[0] * sh[1]);            // ... per output pixel
            }
            cudaFree(buf);
            if (ms < best_ms) {
                best_ms = ms;
                best = std::make_pair(sh[0], sh[1]);
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

bf_status build_state(int n, const bf_plan_t* plans, const float* const* f, float* const* out,
                      BatchState* st, cudaStream_t user)
{
    // ---- images whose radius takes the two-pass FIR run it (its own launches
    // in the graph, after the batched K1 and K2); the others share the queue
    // (two_pass), and so do images whose fused tall tile covers at least a
    // quarter wave of the GPU (a launch of their own fills it as well as the
    // queue would, with the faster tall kernel), and box images of the tall
    // tile's radii (its sliding sums are the form a single execute takes)
    int sms0 = 0;
    if (cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, st->device) != cudaSuccess)
        return BF_ERR_CUDA;
    std::vector<char> two_pass(n, 0);
    for (int i = 0; i < n; ++i) {
        bf_plan_s* p = plans[i];
        const int set_tile = p->opt.t_mode == BF_T_TILE ? p->set_tile : 0;
        const int rows = fwd32t_rows(set_tile) > 0 ? fwd32t_rows(set_tile) : 128;
        const long long tall_ctas = (long long)((p->H + rows - 1) / rows) * ((p->W + 31) / 32);
        two_pass[i] = (p->d_sep_P && set_tile == 0 && !fwd32t_ok(p->R, 0) && sep32_ok(p->R)) ||
                      (fwd32t_ok(p->R, set_tile) && 4 * tall_ctas >= sms0) ||
                      p->opt.plane_dtype != BF_PLANES_FP32 ||
                      forward_args(p, f[i], p->W, out[i], p->W).box_rs ||   // running sums
                      (p->opt.spatial == BF_SPATIAL_BOX && fwd32t_ok(p->R, set_tile));   // sliding sums
    }
    // ---- tile shape per queued image (autotuned per R, remembered per process)
    std::vector<std::pair<int, int>> shape(n);
    for (int i = 0; i < n; ++i) {
        bf_plan_s* p = plans[i];
        if (two_pass[i]) continue;
        auto it = g_tile_choice.find(p->R);
        if (it == g_tile_choice.end()) {
            std::pair<int, int> c = autotune_tile(p, f[i], out[i], user);
            if (!c.first) {
                int th, tw;
                fwd32_tile(p->R, &th, &tw);
                c = std::make_pair(th, tw);
            }
            if (!c.first) return BF_ERR_NOT_SUPPORTED;
            it = g_tile_choice.emplace(p->R, c).first;
        }
        shape[i] = it->second;
    }
    if (cudaStreamSynchronize(user) != cudaSuccess) return BF_ERR_CUDA;

    // ---- host descriptor arrays
    std::vector<RangeImg> rimg;
    std::vector<int4> ritems;
    std::vector<ParamsArgs> pimg(n);
    std::vector<int> bimg, bset;
    std::vector<FwdArgs> fimg(n);
    std::vector<std::pair<int, int>> classes;
    std::vector<std::vector<std::pair<double, int4>>> citems;
    std::vector<int> cmaxR;
    int maxR_range = 0;
    bool range_min = false;          // some image has per-tile T: the min filter runs
    std::vector<unsigned*> zero_T;
    std::vector<int> zero_n;
    std::vector<unsigned long long*> zero_g;
    for (int i = 0; i < n; ++i) {
        bf_plan_s* p = plans[i];
        if (p->opt.t_mode != BF_T_FIXED) {
            RangeImg g;
            g.f = f[i];
            g.pitch = p->W;
            g.H = p->H;
            g.W = p->W;
            g.R = p->R;
            g.set_tile = p->opt.t_mode == BF_T_TILE ? p->set_tile : 0;
            g.sets_x = p->sets_x;
            g.Tbits = p->d_T;
            const int ri = (int)rimg.size();
            rimg.push_back(g);
            for (int by = 0; by < p->H; by += range_tile())
                for (int bx = 0; bx < p->W; bx += range_tile())
                    ritems.push_back(make_int4(ri, by, bx, 0));
            maxR_range = std::max(maxR_range, p->R);
            range_min = range_min || g.set_tile != 0;
            zero_T.push_back(p->d_T);
            zero_n.push_back(p->n_sets);
        }
        zero_g.push_back(p->d_nguard);
        if (p->d_fixcnt) {               // the recheck's list lengths start at zero
            zero_T.push_back(p->d_fixcnt);
            zero_n.push_back(p->n_fixcnt);
        }
        pimg[i] = plan_params_args(p);
        for (int sI = 0; sI < p->n_sets; ++sI) {
            bimg.push_back(i);
            bset.push_back(sI);
        }
        fimg[i] = forward_args(p, f[i], p->W, out[i], p->W);
        if (two_pass[i]) continue;
        int c = -1;
        for (size_t k = 0; k < classes.size(); ++k)
            if (classes[k] == shape[i]) c = (int)k;
        if (c < 0) {
            c = (int)classes.size();
            classes.push_back(shape[i]);
            citems.emplace_back();
            cmaxR.push_back(0);
        }
        cmaxR[c] = std::max(cmaxR[c], p->R);
        // cost bound of one tile: taps x the largest number of terms the plan allows
        const double cost = (2.0 * p->R + 1.0) * (double)p->cap_pairs;
        for (int by = 0; by < p->H; by += shape[i].first)
            for (int bx = 0; bx < p->W; bx += shape[i].second)
                citems[c].push_back(std::make_pair(cost, make_int4(i, by, bx, 0)));
    }
    std::vector<std::vector<int4>> items(classes.size());
    for (size_t c = 0; c < classes.size(); ++c) {
        std::stable_sort(citems[c].begin(), citems[c].end(),
                         [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) {
                             return x.first > y.first;
                         });
        for (auto& e : citems[c]) items[c].push_back(e.second);
    }
    // what the clear kernel zeroes: T words (per image), guard counters, queue heads
    struct Zero {
        unsigned* T;
        int n;
        unsigned long long* g;
    };
    std::vector<Zero> zeros;
    for (size_t k = 0; k < zero_g.size(); ++k) zeros.push_back({nullptr, 0, zero_g[k]});
    for (size_t k = 0; k < zero_T.size(); ++k) zeros.push_back({zero_T[k], zero_n[k], nullptr});
    std::vector<unsigned> heads(classes.size(), 0u);

    // ---- one device blob for all of it
    size_t off = 0;
    const size_t oR = off; off += padded_bytes(rimg);
    const size_t oRI = off; off += padded_bytes(ritems);
    const size_t oP = off; off += padded_bytes(pimg);
    const size_t oBI = off; off += padded_bytes(bimg);
    const size_t oBS = off; off += padded_bytes(bset);
    const size_t oF = off; off += padded_bytes(fimg);
    const size_t oZ = off; off += padded_bytes(zeros);
    const size_t oH = off; off += padded_bytes(heads);
    std::vector<size_t> oI(classes.size());
    for (size_t c = 0; c < classes.size(); ++c) {
        oI[c] = off;
        off += padded_bytes(items[c]);
    }
    if (cudaMalloc(&st->blob, off + 256) != cudaSuccess) return BF_ERR_ALLOC;
    char* d = static_cast<char*>(st->blob);
    bool ok = true;
    auto up = [&](size_t o, const void* src, size_t bytes) {
        if (bytes) ok &= cudaMemcpy(d + o, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    up(oR, rimg.data(), rimg.size() * sizeof(RangeImg));
    up(oRI, ritems.data(), ritems.size() * sizeof(int4));
    up(oP, pimg.data(), pimg.size() * sizeof(ParamsArgs));
    up(oBI, bimg.data(), bimg.size() * sizeof(int));
    up(oBS, bset.data(), bset.size() * sizeof(int));
    up(oF, fimg.data(), fimg.size() * sizeof(FwdArgs));
    up(oZ, zeros.data(), zeros.size() * sizeof(Zero));
    up(oH, heads.data(), heads.size() * sizeof(unsigned));
    for (size_t c = 0; c < classes.size(); ++c) up(oI[c], items[c].data(), items[c].size() * sizeof(int4));
    if (!ok) return BF_ERR_CUDA;

    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, st->device) != cudaSuccess)
        return BF_ERR_CUDA;
    std::vector<int> ctas(classes.size());
    for (size_t c = 0; c < classes.size(); ++c) {
        const int per = fwd32_persistent_ctas_per_sm(classes[c].first, classes[c].second, cmaxR[c]);
        if (per <= 0) return BF_ERR_NOT_SUPPORTED;
        ctas[c] = std::min<int>(sms * per, (int)items[c].size());
    }

    // ---- capture: the per-image launches go to kSide side streams forked
    // from the capture stream after K2 and joined before its end, so that
    // the graph runs them concurrently with each other and with the queue
    constexpr int kSide = 8;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return BF_ERR_CUDA;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
    bool made = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kSide && made; ++k)
        made = cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&join_ev[k], cudaEventDisableTiming) == cudaSuccess;
    auto release = [&]() {
        for (int k = 0; k < kSide; ++k) {
            if (side[k]) cudaStreamDestroy(side[k]);
            if (join_ev[k]) cudaEventDestroy(join_ev[k]);
        }
        if (fork_ev) cudaEventDestroy(fork_ev);
    };
    if (!made) {
        release();
        cudaStreamDestroy(cs);
        return BF_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        e = launch_batch_clear(d + oZ, (int)zeros.size(), reinterpret_cast<unsigned*>(d + oH),
                               (int)heads.size(), cs);
        if (e == cudaSuccess && !ritems.empty())
            e = launch_local_range_batch(reinterpret_cast<const RangeImg*>(d + oR),
                                         reinterpret_cast<const int4*>(d + oRI),
                                         (int)ritems.size(), maxR_range, range_min,
                                         std::min<int>((int)ritems.size(), 4 * sms), cs);
        if (e == cudaSuccess)
            e = launch_params_batch(reinterpret_cast<const ParamsArgs*>(d + oP),
                                    reinterpret_cast<const int*>(d + oBI),
                                    reinterpret_cast<const int*>(d + oBS), (int)bimg.size(), cs);
        if (e == cudaSuccess) e = cudaEventRecord(fork_ev, cs);
        for (int k = 0; k < kSide && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(side[k], fork_ev, 0);
        // own launches, largest images first, round-robin over the side streams
        std::vector<int> own;
        for (int i = 0; i < n; ++i)
            if (two_pass[i]) own.push_back(i);
        std::stable_sort(own.begin(), own.end(), [&](int x, int y) {
            return (long long)plans[x]->H * plans[x]->W * plans[x]->cap_pairs >
                   (long long)plans[y]->H * plans[y]->W * plans[y]->cap_pairs;
        });
        for (size_t j = 0; j < own.size() && e == cudaSuccess; ++j) {
            bf_plan_s* p = plans[own[j]];
            cudaStream_t ss = side[j % kSide];
            if (p->opt.plane_dtype == BF_PLANES_FP32) {
                e = launch_fwd32(fimg[own[j]], ss);
                if (e == cudaSuccess && p->d_fix)      // R > 24: the FP32 recheck
                    e = launch_fixup(fixup_args(p, fimg[own[j]]), p->n_sets, ss);
            } else {
                e = launch_fwd_tc(fimg[own[j]], p->opt.plane_dtype == BF_PLANES_BF16,
                                  p->opt.spin_limit, p->d_status, ss);
                if (e == cudaSuccess && p->d_fix)
                    e = launch_fixup(fixup_args(p, fimg[own[j]]), p->n_sets, ss);
            }
        }
        for (size_t c = 0; c < classes.size() && e == cudaSuccess; ++c)
            e = launch_fwd32_persistent(classes[c].first, classes[c].second, cmaxR[c],
                                        reinterpret_cast<const FwdArgs*>(d + oF),
                                        reinterpret_cast<const int4*>(d + oI[c]),
                                        (int)items[c].size(),
                                        reinterpret_cast<unsigned*>(d + oH) + c, ctas[c], cs);
        // the FP32 recheck of queued images with large windows, after the queue
        for (int i = 0; i < n && e == cudaSuccess; ++i)
            if (!two_pass[i] && plans[i]->d_fix)
                e = launch_fixup(fixup_args(plans[i], fimg[i]), plans[i]->n_sets, cs);
        for (int k = 0; k < kSide && e == cudaSuccess; ++k) {
            e = cudaEventRecord(join_ev[k], side[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, join_ev[k], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&st->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    release();
    cudaStreamDestroy(cs);
    return e == cudaSuccess ? BF_OK : BF_ERR_CUDA;
}

struct ZeroDev {
    unsigned* T;
    int n;
    unsigned long long* g;
};

__global__ void k_batch_clear(const ZeroDev* __restrict__ z, int nz, unsigned* __restrict__ heads,
                              int nh)
{
    for (int i = blockIdx.x; i < nz; i += gridDim.x) {
        const ZeroDev e = z[i];
        if (e.g && threadIdx.x == 0) *e.g = 0ull;
        for (int k = threadIdx.x; k < e.n; k += blockDim.x) e.T[k] = 0u;
    }
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < nh; k += blockDim.x) heads[k] = 0u;
}

}  // namespace

cudaError_t launch_batch_clear(const void* zeros, int n_zeros, unsigned* heads, int n_heads,
                               cudaStream_t s)
{
    const int blocks = std::max(1, std::min(n_zeros, 1024));
    k_batch_clear<<<blocks, 256, 0, s>>>(static_cast<const ZeroDev*>(zeros), n_zeros, heads,
                                         n_heads);
    return cudaGetLastError();
}

namespace bf {

void batch_forget(bf_plan_s* p)
{
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto it = g_states.begin(); it != g_states.end();) {
        bool uses = false;
        for (const void* k : it->first)
            if (k == (const void*)p) uses = true;
        if (uses) {
            free_state(it->second);
            it = g_states.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace bf

extern "C" bf_status bf_execute_batch(int n, const bf_plan_t* plans, const float* const* f,
                                      float* const* out, void* stream)
{
    if (n < 1 || !plans || !f || !out) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !f[i] || !out[i] || (const void*)f[i] == (const void*)out[i])
            return BF_ERR_INVALID_ARG;
        if (plans[i]->device != plans[0]->device) return BF_ERR_INVALID_ARG;
        if (plans[i]->opt.filter != BF_FILTER_FIR || plans[i]->opt.range_kernel != BF_RANGE_COSINE ||
            plans[i]->patch_p)
            return BF_ERR_NOT_SUPPORTED;
    }
    // a plan's workspace (T words, parameter sets, two-pass buffers) serves
    // one image at a time: each image needs a plan of its own
    {
        std::vector<const void*> ps(plans, plans + n);
        std::sort(ps.begin(), ps.end());
        if (std::adjacent_find(ps.begin(), ps.end()) != ps.end()) return BF_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(plans[0]->device) != cudaSuccess) return BF_ERR_CUDA;
    std::vector<const void*> key;
    key.reserve(3 * n);
    for (int i = 0; i < n; ++i) {
        key.push_back(plans[i]);
        key.push_back(f[i]);
        key.push_back(out[i]);
    }
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_states.find(key);
    BatchState* st = nullptr;
    if (it == g_states.end()) {
        st = new BatchState;
        st->key = key;
        st->device = plans[0]->device;
        bf_status rc = build_state(n, plans, f, out, st, s);
        if (rc != BF_OK) {
            free_state(st);
            return rc;
        }
        g_states.emplace(key, st);
    } else {
        st = it->second;
    }
    if (cudaGraphLaunch(st->exec, s) != cudaSuccess) return BF_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        plans[i]->executed = 1;
        plans[i]->last = s;
    }
    return BF_OK;
}
