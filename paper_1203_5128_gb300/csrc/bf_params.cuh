// K2 body (Algorithm 2, steps 3-5) for one parameter set, shared by the
// parameter kernels (bf_params.cu) and the fused per-T-tile range kernel
// (bf_range.cu).
//
// Sec. 1.3: phi(s) = cos(s / (sqrt(N) sigma_r))^N is positive and monotone on
// [-T, T] when N >= N0 = 4 T^2 / (pi^2 sigma_r^2); N = max(1, ceil(N0)).
// eq. (expansion): phi(s) = sum_n w_n cos(omega_n s), w_n = 2^-N C(N, n),
// omega_n = (2n - N) / (sqrt(N) sigma_r).  Sec. 3: keep n = M..N-M with M from
// eq. (trunc) (smallest M with sum_{n<=M+1} w_n > eps/2), eq. (Chernoff)
// (M = (N - sqrt(4 N log(2/eps))) / 2, floored) or the sigma_r bands of
// Algorithm 2 step 4.
//
// Everything here is FP64: 2^-N underflows FP32 from N = 150 and FP64 from
// N = 1075, so the weights are formed in the log domain from a table of
// log(k!) built on the host at plan time.  Terms n and N-n are folded into
// one pair with weight 2 w_n (cos is even); omega is stored as an FP32
// head + tail so that the forward kernel can form omega * f to ~2^-48
// relative.
#pragma once

#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace params {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxTail = 4096;                 // tail weights held for eq. (trunc)
constexpr int kTail = kMaxTail / 2 + 2;        // doubles of tail scratch

__device__ __forceinline__ double log_weight(const ParamsArgs& a, int N, int n)
{
    // same association as a plain reading of log(2^-N C(N, n))
    const double c = a.logfact[N] - (double)N * a.ln2;
    return c - a.logfact[n] - a.logfact[N - n];
}

// One block computes set `set` of `a` (all threads of the block take part);
// tail (kTail doubles) and nm (2 ints) are shared-memory scratch.
__device__ __forceinline__ void params_body(const ParamsArgs& a, int set, double* tail, int* nm)
{
    int& sN = nm[0];
    int& sM = nm[1];
    const double T = (double)a.T[set];

    if (threadIdx.x == 0) {
        const double n0 = (4.0 * T * T) / (kPi * kPi * a.sigma_r * a.sigma_r);
        double c = ceil(n0);
        int N = c < 1.0 ? 1 : (c > 1e9 ? 1000000000 : (int)c);
        sN = N;
    }
    __syncthreads();
    const int N = sN;
    if (N > a.n_cap) {
        if (threadIdx.x == 0) {
            SetHdr h;
            h.N = N; h.M = 0; h.F = -1; h.z = 0; h.w0 = 0.f; h.T = (float)T; h.pad0 = h.pad1 = 0.f;
            a.hdr[set] = h;
            atomicOr(a.status, kDevOrder);
        }
        return;
    }

    // which rule (Algorithm 2 step 4 compares sigma_r on the 8-bit scale)
    int rule = a.rule;
    bool zero_m = !(a.eps > 0.0);
    if (rule == BF_RULE_ALG2 && !zero_m) {
        const double s8 = a.sigma_r * 255.0 / a.value_range;
        if (s8 > 40.0) zero_m = true;
        else if (s8 > 10.0) rule = BF_RULE_TRUNC;
        else rule = BF_RULE_CHERNOFF;
    }

    if (zero_m) {
        if (threadIdx.x == 0) sM = 0;
    } else if (rule == BF_RULE_CHERNOFF) {
        if (threadIdx.x == 0) {
            const double m = 0.5 * ((double)N - sqrt(4.0 * (double)N * log(2.0 / a.eps)));
            int M = (int)floor(m);
            if (M < 0) M = 0;
            if (M > N / 2) M = N / 2;
            sM = M;
        }
    } else {
        // eq. (trunc): tail weights w_0..w_{N/2+1} in parallel, then the running
        // sum in order n = 0, 1, 2, ... on one thread
        const int top = min(N, N / 2 + 1);
        for (int n = threadIdx.x; n <= top; n += blockDim.x) tail[n] = exp(log_weight(a, N, n));
        __syncthreads();
        if (threadIdx.x == 0) {
            int M = 0;
            double S = tail[0];
            for (M = 0; M + 1 <= N; ++M) {
                if (M + 1 > top) break;
                S += tail[M + 1];
                if (S > a.eps / 2.0) break;
            }
            if (M > N / 2) M = N / 2;
            sM = M;
        }
    }
    __syncthreads();
    const int M = sM;
    const int F = (N - M) - N / 2;           // pairs n = floor(N/2)+1 .. N-M
    const double scale = sqrt((double)N) * a.sigma_r;
    Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    for (int k = threadIdx.x; k < F; k += blockDim.x) {
        const int n = N / 2 + 1 + k;
        const double om = (double)(2 * n - N) / scale;
        const double w = exp(log_weight(a, N, n));
        Pair p;
        p.om_hi = (float)om;
        p.om_lo = (float)(om - (double)p.om_hi);
        p.W = (float)(2.0 * w);
        p.pad = 0.f;
        pr[k] = p;
    }
    if (threadIdx.x == 0) {
        SetHdr h;
        h.N = N; h.M = M; h.F = F;
        h.z = (N % 2 == 0) ? 1 : 0;
        h.w0 = h.z ? (float)exp(log_weight(a, N, N / 2)) : 0.f;
        h.T = (float)T;
        h.pad0 = h.pad1 = 0.f;
        a.hdr[set] = h;
    }
}


}  // namespace params
}  // namespace bf
