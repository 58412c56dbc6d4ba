// K1: windowed max / min filter and the dynamic range T.
//
// Sec. 2 of the paper: T = max_x max_{y in window} |f(x-y) - f(x)| (eq.
// (bound)); Prop. 2.1 removes the modulus, Prop. MAX-FILTER and the Appendix
// give the van Herk / Gil-Werman running maxima: split a line into
// partitions of length Wn = 2R+1, take prefix maxima l and suffix maxima r
// inside each partition, and the windowed max at i is max(r[i], l[i+2R]) in
// coordinates padded by R.  Algorithm 1 applies it to rows, then to the
// columns of the row result.
//
// GB300 form: one CTA per 32x32 block of outputs.  The block plus its R halo
// is staged in shared memory once (coalesced), every (line, partition) pair
// is one thread running the two running extrema over its partition, and only
// the entries the combine step reads are kept (r on [0,32), l on
// [2R, 2R+32)), so the line buffers are 32 wide whatever R is.  Max and min
// run in the same pass (padding -inf for the max, +inf for the min).  The
// block's largest local range max(M - f, f - m) goes to its T word with an
// atomicMax on the float's bit pattern (valid: the values are >= 0).
#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kT = 32;       // output block side
constexpr int kThreads = 256;

__device__ __forceinline__ float min_operand(float v)
{
    // out-of-image entries are stored as -inf; they are +inf for the min filter
    return v == -INFINITY ? INFINITY : v;
}

template <bool kImages>
__global__ void __launch_bounds__(kThreads)
k_local_range(const float* __restrict__ f, size_t pitch, int H, int W, int R, int set_tile,
              int sets_x, unsigned* __restrict__ Tbits, float* __restrict__ Mx,
              float* __restrict__ mn)
{
    extern __shared__ float sm[];
    const int L = kT + 2 * R;       // region side
    const int Ls = L + 1;           // padded row stride of the region
    const int Wn = 2 * R + 1;       // window = partition length
    const int P = (L + Wn - 1) / Wn;
    float* reg = sm;                // L x Ls, -inf outside the image
    float* rmax = reg + L * Ls;     // L x 32: row pass, suffix part then result
    float* rmin = rmax + L * kT;
    float* lmax = rmin + L * kT;    // L x 32: row pass, prefix part
    float* lmin = lmax + L * kT;
    float* cRmax = lmin + L * kT;   // 32 x 32 each: column pass
    float* cRmin = cRmax + kT * kT;
    float* cLmax = cRmin + kT * kT;
    float* cLmin = cLmax + kT * kT;
    __shared__ float red[kThreads / 32];

    const int by = blockIdx.y * kT, bx = blockIdx.x * kT;
    const int gy0 = by - R, gx0 = bx - R;
    for (int i = threadIdx.x; i < L * L; i += kThreads) {
        const int r = i / L, c = i - r * L;
        const int gy = gy0 + r, gx = gx0 + c;
        reg[r * Ls + c] = (gy >= 0 && gy < H && gx >= 0 && gx < W)
                              ? __ldg(f + (size_t)gy * pitch + gx) : -INFINITY;
    }
    __syncthreads();

    // ---- rows: running extrema per (row, partition)
    for (int it = threadIdx.x; it < L * P; it += kThreads) {
        const int r = it / P, p = it - r * P;
        const int q0 = p * Wn, q1 = min(q0 + Wn, L);
        const float* row = reg + r * Ls;
        if (q1 > 2 * R && q0 < 2 * R + kT) {       // prefix maxima, kept on [2R, 2R+32)
            float hi = -INFINITY, lo = INFINITY;
            const int qe = min(q1, 2 * R + kT);
            for (int q = q0; q < qe; ++q) {
                const float v = row[q];
                hi = fmaxf(hi, v);
                lo = fminf(lo, min_operand(v));
                if (q >= 2 * R) {
                    lmax[r * kT + (q - 2 * R)] = hi;
                    lmin[r * kT + (q - 2 * R)] = lo;
                }
            }
        }
        if (q0 < kT) {                             // suffix maxima, kept on [0, 32)
            float hi = -INFINITY, lo = INFINITY;
            for (int q = q1 - 1; q >= q0; --q) {
                const float v = row[q];
                hi = fmaxf(hi, v);
                lo = fminf(lo, min_operand(v));
                if (q < kT) {
                    rmax[r * kT + q] = hi;
                    rmin[r * kT + q] = lo;
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L * kT; i += kThreads) {   // combine
        rmax[i] = fmaxf(rmax[i], lmax[i]);
        const float a = rmin[i], b = lmin[i];
        rmin[i] = fminf(a, b);
    }
    __syncthreads();

    // ---- columns of the row result: running extrema per (column, partition)
    for (int it = threadIdx.x; it < kT * P; it += kThreads) {
        const int c = it % kT, p = it / kT;
        const int q0 = p * Wn, q1 = min(q0 + Wn, L);
        if (q1 > 2 * R && q0 < 2 * R + kT) {
            float hi = -INFINITY, lo = INFINITY;
            const int qe = min(q1, 2 * R + kT);
            for (int q = q0; q < qe; ++q) {
                hi = fmaxf(hi, rmax[q * kT + c]);
                lo = fminf(lo, rmin[q * kT + c]);
                if (q >= 2 * R) {
                    cLmax[(q - 2 * R) * kT + c] = hi;
                    cLmin[(q - 2 * R) * kT + c] = lo;
                }
            }
        }
        if (q0 < kT) {
            float hi = -INFINITY, lo = INFINITY;
            for (int q = q1 - 1; q >= q0; --q) {
                hi = fmaxf(hi, rmax[q * kT + c]);
                lo = fminf(lo, rmin[q * kT + c]);
                if (q < kT) {
                    cRmax[q * kT + c] = hi;
                    cRmin[q * kT + c] = lo;
                }
            }
        }
    }
    __syncthreads();

    // ---- local range and its block maximum
    float best = 0.0f;
    for (int i = threadIdx.x; i < kT * kT; i += kThreads) {
        const int oy = i / kT, ox = i - oy * kT;
        const int gy = by + oy, gx = bx + ox;
        if (gy >= H || gx >= W) continue;
        const float M = fmaxf(cRmax[i], cLmax[i]);
        const float m = fminf(cRmin[i], cLmin[i]);
        const float v = reg[(oy + R) * Ls + (ox + R)];
        if (kImages) {
            Mx[(size_t)gy * pitch + gx] = M;
            mn[(size_t)gy * pitch + gx] = m;
        } else {
            best = fmaxf(best, fmaxf(M - v, v - m));
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

size_t range_smem(int R)
{
    const size_t L = kT + 2 * (size_t)R;
    return sizeof(float) * (L * (L + 1) + 4 * L * kT + 4 * kT * kT);
}

template <bool kImages>
cudaError_t launch(const float* f, size_t pitch, int H, int W, int R, int set_tile, int sets_x,
                   unsigned* Tbits, float* Mx, float* mn, cudaStream_t s)
{
    const size_t smem = range_smem(R);
    cudaError_t e = cudaFuncSetAttribute(k_local_range<kImages>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT);
    k_local_range<kImages><<<grid, kThreads, smem, s>>>(f, pitch, H, W, R, set_tile, sets_x,
                                                        Tbits, Mx, mn);
    return cudaGetLastError();
}

}  // namespace

int range_max_radius()
{
    int R = 0;
    while (range_smem(R + 1) <= 226 * 1024) ++R;   // static reduction buffer rides on top
    return R;
}

cudaError_t launch_local_range(const float* f, size_t pitch, int H, int W, int R, int set_tile,
                               int sets_x, unsigned* Tbits, cudaStream_t s)
{
    return launch<false>(f, pitch, H, W, R, set_tile, sets_x, Tbits, nullptr, nullptr, s);
}

cudaError_t launch_maxmin(const float* f, size_t pitch, int H, int W, int R, float* Mx, float* mn,
                          cudaStream_t s)
{
    return launch<true>(f, pitch, H, W, R, 0, 1, nullptr, Mx, mn, s);
}

}  // namespace bf
