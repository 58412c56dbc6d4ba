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

#include "bf_internal.cuh"

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

}  // namespace

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
