// K1: windowed max / min filter and the dynamic range T.
//
// Sec. 2 of the paper: T = max_x max_{y in window} |f(x-y) - f(x)| (eq.
// (bound)); Prop. 2.1 removes the modulus (for the image-wide T the max
// filter alone suffices: max_x (M(x) - f(x)) = max_x (f(x) - m(x))), Prop.
// MAX-FILTER and the Appendix give the van Herk / Gil-Werman running maxima:
// split a line into partitions of length Wn = 2R+1, take suffix maxima r and
// prefix maxima l inside each partition, and the windowed max of the window
// starting at i is max(r[i], l[i+2R]).  Algorithm 1 applies it to rows, then
// to the columns of the row result.
//
// GB300 form: one CTA of 1024 threads per 64 x 64 block of outputs, two CTAs
// per SM (their serial partition chains are latency-bound, so the more warps
// the better: 256 threads took 0.28 ms at 4096^2, 1024 threads 0.215 ms).  The block plus its R
// halo is staged in shared memory once (coalesced, by cp.async so that a
// thread's copies are all in flight together).  Each (line, partition)
// is one thread running the partition's suffix (then prefix) maxima
// sequentially -- 3 max operations per point as in the Appendix -- with the
// 32 lanes of a warp on 32 consecutive lines, so every step is one
// conflict-free shared load per lane and the loops carry no branches.  Only
// the entries the combine reads are kept: suffix maxima on [0, 64) are
// written first, then the prefix maxima on [2R, 2R+64) are folded in.
// Per-tile T needs max and min (each (line, partition) then gives a max item
// and a min item, run by different threads); the image-wide T needs only the
// max (Prop. 2.1).  The block's largest local range goes to its T word with an
// atomicMax on the float's bit pattern (valid: the values are >= 0).
#include <math.h>

#include "bf_params.cuh"

namespace bf {
namespace {

constexpr int kT = 64;          // output block side
constexpr int kTp = kT + 1;     // padded row stride of the 64-wide buffers
constexpr int kThreads = 1024;  // two CTAs per SM: 64 warps to hide the serial partition chains

__device__ __forceinline__ float min_operand(float v)
{
    // out-of-image entries are stored as -inf; they are +inf for the min filter
    return v == -INFINITY ? INFINITY : v;
}

// Suffix maxima (kIsMin: minima) of src[q0..q1), stride `st` between
// entries, written to dst[q * dst_st] for q < lim.
template <bool kIsMin>
__device__ __forceinline__ void suffix_part(const float* src, int st, int q0, int q1, int lim,
                                            float* dst, int dst_st)
{
    float acc = kIsMin ? INFINITY : -INFINITY;
    int q = q1 - 1;
    const int qs = min(q1, lim);          // entries below qs are stored
#pragma unroll 4
    for (; q >= qs; --q)
        acc = kIsMin ? fminf(acc, min_operand(src[q * st])) : fmaxf(acc, src[q * st]);
#pragma unroll 4
    for (; q >= q0; --q) {
        acc = kIsMin ? fminf(acc, min_operand(src[q * st])) : fmaxf(acc, src[q * st]);
        dst[q * dst_st] = acc;
    }
}

// Prefix maxima (minima) of src[q0..qe), folded into dst[(q - off) * dst_st]
// for q >= off: the combine max(r[i], l[i + 2R]) of the Appendix.
template <bool kIsMin>
__device__ __forceinline__ void prefix_part(const float* src, int st, int q0, int qe, int off,
                                            float* dst, int dst_st)
{
    float acc = kIsMin ? INFINITY : -INFINITY;
    int q = q0;
    const int qs = max(q0, off);
#pragma unroll 4
    for (; q < qs; ++q)
        acc = kIsMin ? fminf(acc, min_operand(src[q * st])) : fmaxf(acc, src[q * st]);
#pragma unroll 4
    for (; q < qe; ++q) {
        acc = kIsMin ? fminf(acc, min_operand(src[q * st])) : fmaxf(acc, src[q * st]);
        float* d = dst + (q - off) * dst_st;
        *d = kIsMin ? fminf(*d, acc) : fmaxf(*d, acc);
    }
}

// One 64 x 64 output block with origin (by, bx): the whole block takes part.
template <bool kMin, bool kImages>
__device__ __forceinline__ void range_body(const float* __restrict__ f, size_t pitch, int H, int W,
                                           int R, int set_tile, int sets_x,
                                           unsigned* __restrict__ Tbits, float* __restrict__ Mx,
                                           float* __restrict__ mn, int by, int bx, float* sm,
                                           float* red)
{
    const int L = kT + 2 * R;       // region side (even)
    const int Ls = L + 1;           // odd row stride: lanes on consecutive rows hit distinct banks
    const int Wn = 2 * R + 1;       // window = partition length
    const int P = (L + Wn - 1) / Wn;
    // reg (L x Ls, -inf outside the image) is dead after the row pass, so the
    // column pass result (kT x kTp per filter) is written over it
    const int reg_floats = max(L * Ls, (kMin ? 2 : 1) * kT * kTp);
    float* reg = sm;
    float* rmax = reg + reg_floats;  // L x kTp: row pass result
    float* rmin = rmax + L * kTp;
    float* cmax = reg;               // kT x kTp: column pass result
    float* cmin = cmax + kT * kTp;

    // stage the block + halo: in-image entries by cp.async (all of a thread's
    // copies in flight at once), -inf elsewhere
    const int gy0 = by - R, gx0 = bx - R;
    for (int r = threadIdx.x / 32; r < L; r += kThreads / 32) {
        const int gy = gy0 + r;
        const bool rin = gy >= 0 && gy < H;
        for (int c = threadIdx.x % 32; c < L; c += 32) {
            const int gx = gx0 + c;
            float* dst = reg + r * Ls + c;
            if (rin && gx >= 0 && gx < W)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                             ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                               "l"(f + (size_t)gy * pitch + gx)
                             : "memory");
            else
                *dst = -INFINITY;
        }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    // ---- rows: suffix parts (partitions meeting [0, kT)), then prefix parts
    //      (partitions meeting [2R, 2R + kT)); lane = row.  With the min filter
    //      the max and min of a (line, partition) are separate items, so that
    //      every phase spreads over more of the block's threads.
    constexpr int NF = kMin ? 2 : 1;
    const int pr_hi = (kT - 1) / Wn;              // last partition meeting [0, kT)
    const int pl_lo = (2 * R) / Wn, pl_hi = (2 * R + kT - 1) / Wn;
    const int nrs = L * (pr_hi + 1);
    for (int it = threadIdx.x; it < NF * nrs; it += kThreads) {
        const bool mn_item = kMin && it >= nrs;
        const int jt = mn_item ? it - nrs : it;
        const int p = jt / L, r = jt - p * L;
        const int q0 = p * Wn, q1 = min(q0 + Wn, L);
        if (mn_item) suffix_part<true>(reg + r * Ls, 1, q0, q1, kT, rmin + r * kTp, 1);
        else suffix_part<false>(reg + r * Ls, 1, q0, q1, kT, rmax + r * kTp, 1);
    }
    __syncthreads();
    const int nrp = L * (pl_hi - pl_lo + 1);
    for (int it = threadIdx.x; it < NF * nrp; it += kThreads) {
        const bool mn_item = kMin && it >= nrp;
        const int jt = mn_item ? it - nrp : it;
        const int p = pl_lo + jt / L, r = jt % L;
        const int q0 = p * Wn, qe = min(min(q0 + Wn, L), 2 * R + kT);
        if (mn_item) prefix_part<true>(reg + r * Ls, 1, q0, qe, 2 * R, rmin + r * kTp, 1);
        else prefix_part<false>(reg + r * Ls, 1, q0, qe, 2 * R, rmax + r * kTp, 1);
    }
    __syncthreads();

    // ---- columns of the row result; lane = column
    const int ncs = kT * (pr_hi + 1);
    for (int it = threadIdx.x; it < NF * ncs; it += kThreads) {
        const bool mn_item = kMin && it >= ncs;
        const int jt = mn_item ? it - ncs : it;
        const int p = jt / kT, c = jt % kT;
        const int q0 = p * Wn, q1 = min(q0 + Wn, L);
        if (mn_item) suffix_part<true>(rmin + c, kTp, q0, q1, kT, cmin + c, kTp);
        else suffix_part<false>(rmax + c, kTp, q0, q1, kT, cmax + c, kTp);
    }
    __syncthreads();
    const int ncp = kT * (pl_hi - pl_lo + 1);
    for (int it = threadIdx.x; it < NF * ncp; it += kThreads) {
        const bool mn_item = kMin && it >= ncp;
        const int jt = mn_item ? it - ncp : it;
        const int p = pl_lo + jt / kT, c = jt % kT;
        const int q0 = p * Wn, qe = min(min(q0 + Wn, L), 2 * R + kT);
        if (mn_item) prefix_part<true>(rmin + c, kTp, q0, qe, 2 * R, cmin + c, kTp);
        else prefix_part<false>(rmax + c, kTp, q0, qe, 2 * R, cmax + c, kTp);
    }
    __syncthreads();
    (void)P;

    // ---- local range and its block maximum
    float best = 0.0f;
    for (int i = threadIdx.x; i < kT * kT; i += kThreads) {
        const int oy = i / kT, ox = i - oy * kT;
        const int gy = by + oy, gx = bx + ox;
        if (gy >= H || gx >= W) continue;
        const float M = cmax[oy * kTp + ox];
        const float v = __ldg(f + (size_t)gy * pitch + gx);
        if (kImages) {
            Mx[(size_t)gy * pitch + gx] = M;
            mn[(size_t)gy * pitch + gx] = cmin[oy * kTp + ox];
        } else {
            best = fmaxf(best, M - v);
            if (kMin) best = fmaxf(best, v - cmin[oy * kTp + ox]);
        }
    }
    if (!kImages) {
        for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = 0.0f;
            for (int w = 0; w < kThreads / 32; ++w) b = fmaxf(b, red[w]);
            const int set = set_tile ? (by / set_tile) * sets_x + (bx / set_tile) : 0;
            atomicMax(Tbits + set, __float_as_uint(b));
        }
    }
}

template <bool kMin, bool kImages>
__global__ void __launch_bounds__(kThreads, 2)
k_local_range(const float* __restrict__ f, size_t pitch, int H, int W, int R, int set_tile,
              int sets_x, unsigned* __restrict__ Tbits, float* __restrict__ Mx,
              float* __restrict__ mn, int by0)
{
    extern __shared__ float sm[];
    __shared__ float red[kThreads / 32];
    range_body<kMin, kImages>(f, pitch, H, W, R, set_tile, sets_x, Tbits, Mx, mn,
                              (by0 + (int)blockIdx.y) * kT, blockIdx.x * kT, sm, red);
}

// Batched: CTAs stride over (image, block row, block column) items; the min
// filter runs for images with per-tile T only (Prop. 2.1: the image-wide T
// needs the max filter alone).
__global__ void __launch_bounds__(kThreads)
k_local_range_batch(const RangeImg* __restrict__ imgs, const int4* __restrict__ items, int n_items)
{
    extern __shared__ float sm[];
    __shared__ float red[kThreads / 32];
    for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
        const int4 it = items[i];
        const RangeImg g = imgs[it.x];
        __syncthreads();
        if (g.set_tile)
            range_body<true, false>(g.f, g.pitch, g.H, g.W, g.R, g.set_tile, g.sets_x, g.Tbits,
                                    nullptr, nullptr, it.y, it.z, sm, red);
        else
            range_body<false, false>(g.f, g.pitch, g.H, g.W, g.R, 0, 1, g.Tbits, nullptr, nullptr,
                                     it.y, it.z, sm, red);
    }
}

size_t range_smem(int R, bool with_min)
{
    const size_t L = kT + 2 * (size_t)R;
    const size_t lines = with_min ? 2 : 1;
    const size_t reg = L * (L + 1) > lines * kT * kTp ? L * (L + 1) : lines * kT * kTp;
    return sizeof(float) * (reg + lines * L * kTp);
}

template <bool kMin, bool kImages>
cudaError_t launch(const float* f, size_t pitch, int H, int W, int R, int set_tile, int sets_x,
                   unsigned* Tbits, float* Mx, float* mn, cudaStream_t s, int by0 = 0, int nby = 0)
{
    const size_t smem = range_smem(R, kMin);
    cudaError_t e = cudaFuncSetAttribute(k_local_range<kMin, kImages>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kT - 1) / kT, nby > 0 ? nby : (H + kT - 1) / kT);
    k_local_range<kMin, kImages><<<grid, kThreads, smem, s>>>(f, pitch, H, W, R, set_tile, sets_x,
                                                              Tbits, Mx, mn, by0);
    return cudaGetLastError();
}

// ---- fused per-T-tile form: T of one T-tile and its parameter set ---------
//
// One CTA of 1024 threads per S x S T-tile: the tile plus its R halo is
// staged once (NaN outside the image, which fmaxf / fminf skip, so no
// select), then, for 64 output columns at a time, a row pass and a column
// pass give the windowed max M and min m, and the CTA reduces max(M - f,
// f - m) over the tile's pixels into T (exact: max, min and one rounded
// difference, rounding being monotone).  Each pass item is one line and 8
// consecutive outputs: the 2R+1 windows of 8 neighbours share their middle
// 2R - 6 inputs, so an item takes that core's max and min once, the suffix
// extremes of the 7 inputs before it and the prefix extremes of the 7 after
// it, and combines (about 2R + 8 loads and 4R + 40 max / min operations for
// 16 results, against 3 operations per point and pass for van Herk but with
// no serial chain).  Then the same CTA computes the set's N, M and pair
// table (Algorithm 2, steps 3-5), its shared memory reused as scratch.
constexpr int kTP = 1024;
constexpr int kTC = 64;            // output columns per row-pass chunk
constexpr int kTCs = kTC + 1;      // their row stride: the row pass's lanes (rows) hit distinct banks

// max (kMax) and/or min (kMin) of the 8 windows [x0 + i, x0 + i + 2R], i =
// 0..7, of a line with stride st (R >= 4: the windows share [x0 + 7, x0 +
// 2R], whose extremes are taken with four independent accumulators)
template <bool kMax, bool kMin>
__device__ __forceinline__ void window8(const float* v, int st, int R, float* mx, float* mn)
{
    const int w = 2 * R;
    if (R < 4) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float a = -INFINITY, b = INFINITY;
            for (int k = 0; k <= w; ++k) {
                const float x = v[(i + k) * st];
                if (kMax) a = fmaxf(a, x);
                if (kMin) b = fminf(b, x);
            }
            if (kMax) mx[i] = a;
            if (kMin) mn[i] = b;
        }
        return;
    }
    float ca[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    float cb[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
    int k = 7;
    for (; k + 3 <= w; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float x = v[(k + u) * st];
            if (kMax) ca[u] = fmaxf(ca[u], x);
            if (kMin) cb[u] = fminf(cb[u], x);
        }
    }
    for (; k <= w; ++k) {
        const float x = v[k * st];
        if (kMax) ca[0] = fmaxf(ca[0], x);
        if (kMin) cb[0] = fminf(cb[0], x);
    }
    const float cA = fmaxf(fmaxf(ca[0], ca[1]), fmaxf(ca[2], ca[3]));
    const float cB = fminf(fminf(cb[0], cb[1]), fminf(cb[2], cb[3]));
    float lv[7], rv[7];                        // the 7 inputs before and after the core
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        lv[i] = v[i * st];
        rv[i] = v[(w + 1 + i) * st];
    }
    float la = -INFINITY, lb = INFINITY;       // suffix extremes of v[i .. 6]
    float lA[8], lB[8];
    lA[7] = -INFINITY;
    lB[7] = INFINITY;
#pragma unroll
    for (int i = 6; i >= 0; --i) {
        if (kMax) la = fmaxf(la, lv[i]);
        if (kMin) lb = fminf(lb, lv[i]);
        lA[i] = la;
        lB[i] = lb;
    }
    float ra = -INFINITY, rb = INFINITY;       // prefix extremes of v[w + 1 .. w + i]
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i > 0) {
            if (kMax) ra = fmaxf(ra, rv[i - 1]);
            if (kMin) rb = fminf(rb, rv[i - 1]);
        }
        if (kMax) mx[i] = fmaxf(fmaxf(lA[i], cA), ra);
        if (kMin) mn[i] = fminf(fminf(lB[i], cB), rb);
    }
}

__global__ void __launch_bounds__(kTP, 1)
k_tile_params(const float* __restrict__ f, size_t pitch, int H, int W, int R, int S, int sets_x,
              int set0, unsigned* __restrict__ Tbits, ParamsArgs pa)
{
    extern __shared__ float sm[];
    __shared__ float red[kTP / 32];
    const int L = S + 2 * R, Ls = L + 1;          // odd stride: lanes on rows hit distinct banks
    float* reg = sm;                              // L x Ls
    float* bmx = reg + (size_t)L * Ls;            // L x kTCs row-pass max
    float* bmn = bmx + (size_t)L * kTCs;          // L x kTCs row-pass min
    const int set = set0 + blockIdx.x;
    const int ty = set / sets_x, tx = set - ty * sets_x;
    const int gy0 = ty * S - R, gx0 = tx * S - R;
    const int tid = threadIdx.x;

    // stage the tile + halo: in-image entries by cp.async (every copy of a
    // thread in flight at once), NaN elsewhere
    for (int r = tid >> 5; r < L; r += kTP / 32) {
        const int gy = gy0 + r;
        const bool rin = gy >= 0 && gy < H;
        for (int c = tid & 31; c < L; c += 32) {
            const int gx = gx0 + c;
            float* dst = reg + r * Ls + c;
            if (rin && gx >= 0 && gx < W)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                             ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                               "l"(f + (size_t)gy * pitch + gx)
                             : "memory");
            else
                *dst = __int_as_float(0x7fc00000);
        }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    float best = 0.0f;
    for (int c0 = 0; c0 < S; c0 += kTC) {
        // rows: item (r, g) -> outputs c0 + 8g .. c0 + 8g + 7 of region row r
        for (int it = tid; it < L * (kTC / 8); it += kTP) {
            const int r = it % L, g = it / L;
            float mx[8], mn[8];
            window8<true, true>(reg + r * Ls + c0 + 8 * g, 1, R, mx, mn);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                bmx[r * kTCs + 8 * g + i] = mx[i];
                bmn[r * kTCs + 8 * g + i] = mn[i];
            }
        }
        __syncthreads();
        // columns: item (c, g) -> output rows 8g .. 8g + 7 of chunk column c
        for (int it = tid; it < kTC * (S / 8); it += kTP) {
            const int c = it % kTC, g = it / kTC;
            float mx[8], mn[8];
            window8<true, false>(bmx + (8 * g) * kTCs + c, kTCs, R, mx, nullptr);
            window8<false, true>(bmn + (8 * g) * kTCs + c, kTCs, R, nullptr, mn);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float v = reg[(8 * g + i + R) * Ls + c0 + c + R];   // NaN outside
                best = fmaxf(best, fmaxf(mx[i] - v, v - mn[i]));
            }
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((tid & 31) == 0) red[tid >> 5] = best;
    __syncthreads();
    if (tid == 0) {
        float b = 0.0f;
        for (int w = 0; w < kTP / 32; ++w) b = fmaxf(b, red[w]);
        Tbits[set] = __float_as_uint(b);
    }
    __syncthreads();
    // Algorithm 2, steps 3-5 for this set; the staging memory is free now
    params::params_body(pa, set, reinterpret_cast<double*>(sm),
                        reinterpret_cast<int*>(sm + 2 * params::kTail));
}

size_t tile_params_smem(int R, int S)
{
    const size_t L = (size_t)S + 2 * (size_t)R;
    const size_t st = sizeof(float) * (L * (L + 1) + 2 * L * kTCs);
    const size_t pr = sizeof(double) * params::kTail + 2 * sizeof(int);
    return st > pr ? st : pr;
}

}  // namespace

bool tile_params_ok(int R, int set_tile, int n_cap)
{
    return set_tile > 0 && set_tile % kTC == 0 && n_cap <= params::kMaxTail &&
           tile_params_smem(R, set_tile) + sizeof(float) * (kTP / 32) <= 227 * 1024;
}

cudaError_t launch_tile_params(const float* f, size_t pitch, int H, int W, int R, int set_tile,
                               int sets_x, int set0, int n_sets, unsigned* Tbits,
                               const ParamsArgs& pa, cudaStream_t s)
{
    const size_t smem = tile_params_smem(R, set_tile);
    cudaError_t e = cudaFuncSetAttribute(k_tile_params,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tile_params<<<n_sets, kTP, smem, s>>>(f, pitch, H, W, R, set_tile, sets_x, set0, Tbits, pa);
    return cudaGetLastError();
}

int range_tile() { return kT; }

size_t range_smem_bytes(int R) { return range_smem(R, true); }

cudaError_t launch_local_range_batch(const RangeImg* imgs, const int4* items, int n_items,
                                     int max_R, bool with_min, int n_ctas, cudaStream_t s)
{
    const size_t smem = range_smem(max_R, with_min);
    cudaError_t e = cudaFuncSetAttribute(k_local_range_batch,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_local_range_batch<<<n_ctas, kThreads, smem, s>>>(imgs, items, n_items);
    return cudaGetLastError();
}

int range_max_radius()
{
    int R = 0;
    while (range_smem(R + 1, true) <= 226 * 1024) ++R;   // static reduction buffer rides on top
    return R;
}

cudaError_t launch_local_range(const float* f, size_t pitch, int H, int W, int R, int set_tile,
                               int sets_x, unsigned* Tbits, cudaStream_t s, int by0, int nby)
{
    // per-tile T needs the min filter too; the image-wide T does not (Prop. 2.1)
    if (set_tile)
        return launch<true, false>(f, pitch, H, W, R, set_tile, sets_x, Tbits, nullptr, nullptr, s,
                                   by0, nby);
    return launch<false, false>(f, pitch, H, W, R, 0, 1, Tbits, nullptr, nullptr, s);
}

cudaError_t launch_maxmin(const float* f, size_t pitch, int H, int W, int R, float* Mx, float* mn,
                          cudaStream_t s)
{
    return launch<true, true>(f, pitch, H, W, R, 0, 1, nullptr, Mx, mn, s);
}

}  // namespace bf
