// FP32 recheck of the outputs that a 16-bit-plane forward (K3-tc) listed.
//
// At a pixel unlike most of its window the denominator of eq. (f2) is a
// small part of the window's spatial mass, and the terms that cancel down to
// it are of the order of that mass: the 16-bit rounding of the modulated
// planes (and of the vertical pass) is amplified by mass / den.  K3-tc lists
// every output with den < kappa * (g * 1_Omega)(x); this kernel recomputes
// each of them in FP32 by the direct sum of eq. (BF) with the pixel's own
// phi_eps (eq. (approx), the same N, M and folded weights as the planes):
//
//   out(x) = f(x) + sum_y g(x - y) phi_eps(d_y) d_y / sum_y g(x - y) phi_eps(d_y),
//   d_y = f(y) - f(x),   phi_eps(d) = w0 [N even] + sum_k W_k cos(omega_k d),
//
// with omega_k = omega_0 + k Delta, Delta = 2 / (sqrt(N) sigma_r) (omega_0 =
// Delta for even N, Delta / 2 for odd N).  The pair sum is the real part of
// e^{i omega_0 d} P(z), P(z) = sum_k W_k z^k, z = e^{i Delta d}, evaluated by
// Horner's rule on the unit circle (4 FMA-pipe operations per term, no
// rounding growth beyond K ulps); d is formed exactly as a head + tail
// (two-sum) and Delta d as a head + tail product, and |Delta d| <= pi
// whenever |d| <= T (N >= 4 T^2 / (pi^2 sigma_r^2)), so one accurate sincosf
// per neighbour gives z.  num and den are compensated sums (two-sum per
// term), then the denominator guard and the normalisation of the forward.
//
// One warp per listed pixel (lanes over the (2R+1)^2 window); the list length
// is read on the device, so the launch needs no host synchronisation.
#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr int kCtasPerSm = 8;

// s + c += v, c collecting the rounding error of each addition (two-sum)
__device__ __forceinline__ void comp_add(float& s, float& c, float v)
{
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

__global__ void __launch_bounds__(kThreads) k_fixup(FixArgs a)
{
    extern __shared__ float sm[];
    const int RW = 2 * a.R + 1;
    float* taps = sm;                                       // 2R+1
    float* wk = sm + ((RW + 3) & ~3) + (threadIdx.x >> 5) * a.cap_pairs;
    for (int i = threadIdx.x; i < RW; i += kThreads) taps[i] = a.taps[i];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const unsigned gw = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const unsigned nw = (gridDim.x * kThreads) >> 5;
    const unsigned n = *a.count;
    const float full = full_mass(taps, a.R);
    for (unsigned e = gw; e < n; e += nw) {
        const unsigned idx = a.list[e];
        const int gy = (int)(idx / (unsigned)a.W), gx = (int)(idx - (unsigned)gy * a.W);
        const int set = a.set_tile ? (gy / a.set_tile) * a.sets_x + gx / a.set_tile : 0;
        const SetHdr hd = a.hdr[set];
        const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
        const int K = hd.F;
        __syncwarp();
        for (int k = lane; k < K; k += 32) wk[k] = pr[k].W;
        __syncwarp();
        const double D = 2.0 / (sqrt((double)hd.N) * a.sigma_r);
        const float Dhi = (float)D, Dlo = (float)(D - (double)Dhi);
        const bool odd = hd.N & 1;
        const float w0 = hd.z ? hd.w0 : 0.f;
        const float fx = a.f[(size_t)gy * a.f_pitch + gx];

        float ns = 0.f, nc = 0.f, ds = 0.f, dc = 0.f;
        for (int p = lane; p < RW * RW; p += 32) {
            const int iy = p / RW, ix = p - iy * RW;
            const int y = gy + iy - a.R, x = gx + ix - a.R;
            if (y < 0 || y >= a.H || x < 0 || x >= a.W) continue;
            const float fy = a.f[(size_t)y * a.f_pitch + x];
            // d = fy - fx = dh + dl exactly
            const float dh = fy - fx;
            const float t = dh - fy;
            const float dl = (fy - (dh - t)) + (-fx - t);
            // Delta * d (half of it for odd N) as head + tail
            const float ph = Dhi * dh;
            float pe = fmaf(Dhi, dh, -ph);
            pe = fmaf(Dhi, dl, pe);
            pe = fmaf(Dlo, dh, pe);
            float ang = ph + pe;
            if (odd) ang *= 0.5f;
            float s1, c1;
            sincosf(ang, &s1, &c1);
            const float mr = c1, mi = s1;                      // e^{i omega_0 d}
            const float zr = odd ? fmaf(c1, c1, -s1 * s1) : c1;
            const float zi = odd ? 2.f * c1 * s1 : s1;         // e^{i Delta d}
            // P(z) by Horner from the highest term
            float pr_ = 0.f, pi_ = 0.f;
            for (int k = K - 1; k >= 0; --k) {
                const float tr = fmaf(-pi_, zi, fmaf(pr_, zr, wk[k]));
                pi_ = fmaf(pr_, zi, pi_ * zr);
                pr_ = tr;
            }
            const float phi = fmaf(mr, pr_, -mi * pi_) + w0;
            const float wgt = taps[iy] * taps[ix] * phi;
            comp_add(ds, dc, wgt);
            comp_add(ns, nc, wgt * dh);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float ns2 = __shfl_xor_sync(0xffffffffu, ns, off);
            const float nc2 = __shfl_xor_sync(0xffffffffu, nc, off);
            const float ds2 = __shfl_xor_sync(0xffffffffu, ds, off);
            const float dc2 = __shfl_xor_sync(0xffffffffu, dc, off);
            comp_add(ns, nc, ns2);
            nc += nc2;
            comp_add(ds, dc, ds2);
            dc += dc2;
        }
        if (lane == 0) {
            const float num = ns + nc, den = ds + dc;
            const float rmass = clipped_mass(taps, a.R, gy, a.H, full);
            const float cmass = clipped_mass(taps, a.R, gx, a.W, full);
            float v;
            if (den > kGuard * rmass * cmass) {
                v = fx + __fdiv_rn(num, den);
            } else {
                v = fx;
                atomicAdd(a.n_guarded, 1ull);
            }
            a.out[(size_t)gy * a.out_pitch + gx] = v;
        }
    }
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    }
    return n;
}

}  // namespace

cudaError_t launch_fixup(const FixArgs& a, cudaStream_t s)
{
    const int RW = 2 * a.R + 1;
    const size_t smem = sizeof(float) * (((RW + 3) & ~3) + (size_t)kWarps * a.cap_pairs);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fixup, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_fixup<<<sm_count() * kCtasPerSm, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bf
