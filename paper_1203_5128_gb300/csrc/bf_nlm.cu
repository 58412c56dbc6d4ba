// O(1) non-local means with a small patch (Sec. 6, eqs. (NL1), (NL2)).
//
// The range kernel acts on the p pixels u_1 = 0, u_2, ..., u_p of a patch:
// g(s_1, ..., s_p) = prod_i g_r(s_i), s_i = f(x + u_i) - f(x - y + u_i), each
// one-dimensional Gaussian replaced by phi_eps (eq. (approx)) with the N and
// M that T (eq. (bound), Algorithm 1) and Algorithm 2 give (every s_i lies
// in [-T, T]: both pixels are within R of each other).  Expanding each
// phi_eps(s_i) = sum_n w_n exp(j omega_n s_i) (n = M .. N - M) turns the
// product into a sum over multi-indices nu = (n_1, ..., n_p) of weight
// w_nu = prod_i w_{n_i} and phase theta_nu(z) = sum_i omega_{n_i} f(z + u_i):
//
//   NL2(x) = sum_nu w_nu [cos theta_nu(x) (s * cos theta_nu)(x) + sin theta_nu(x) (s * sin theta_nu)(x)]
//   NL1(x) = the same with the planes f cos theta_nu, f sin theta_nu,
//
// out = NL1 / NL2: the bilateral filter's shiftable form with a phase that
// reads the whole patch.  nu and its mirror (every n_i -> N - n_i) give
// conjugate terms, so only the first half of the K^p multi-indices (K = N -
// 2M + 1) runs, with weight 2 w_nu (the self-mirror middle one, for odd
// K^p, with w_nu).  Patch values outside the image are taken at the nearest
// in-image pixel; the spatial sums are clipped to the image as everywhere.
//
// GB300 form: the FP32 fused tile of the bilateral forward (fir32 row and
// column passes); per term every halo pixel gets its patch phase as an FP32
// head + exact tail (TwoProduct per patch pixel), reduced by 2 pi in two
// parts and evaluated on the SFU, with f centred on c0 = value_range / 2 (a
// constant phase shift per term, which cancels between the modulation and
// the demodulation).
#include <math.h>

#include "bf_fir32.cuh"

namespace bf {
namespace {

using fir32::Geo;

constexpr int kMaxPatch = 9;

// s + c += v, c collecting the rounding error of each addition (two-sum):
// num and den sum up to (K^p + 1) / 2 terms (about 10^5 for a 5-pixel patch)
__device__ __forceinline__ void comp_add(float& s, float& c, float v)
{
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

template <int TH, int TW>
__global__ void __launch_bounds__(TH * TW / 8) k_nlm32(FwdArgs a, NlmPatch pt)
{
    constexpr int NT = TH * TW / 8;
    constexpr int NW = NT / 32;
    extern __shared__ float sm[];
    const Geo G(a.R, TH, TW);
    const int R = a.R;
    const int EW = G.RWp + 2;                      // patch-extended region row stride
    const size_t reg = (size_t)G.RH * G.RWp;
    float* fext = sm;                              // (RH + 2) x EW, centred f, clamped coords
    float* fsm = fext + (size_t)(G.RH + 2) * EW;   // RH x RWp centred f, 0 outside the image
    float* csm = fsm + reg;
    float* ssm = csm + reg;
    float* hsm = ssm + reg;                        // 4 x RHp x TW
    float* gz = hsm + 4 * (size_t)G.RHp * TW;
    float* tw_ = gz + G.ngz;                       // per kept index: om_hi, om_lo, w
    const size_t hplane = (size_t)G.RHp * TW;

    const int by = blockIdx.y * TH, bx = blockIdx.x * TW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gy0 = by - R, gx0 = bx - R;
    const SetHdr hd = a.hdr[0];
    const int o = tid % TW, rb = tid / TW;
    const int gx = bx + o;

    if (hd.F < 0) {          // order above the cap: pass the image through
        for (int i = 0; i < 8; ++i) {
            const int gy = by + rb * 8 + i;
            if (gy < a.H && gx < a.W)
                a.out[(size_t)gy * a.out_pitch + gx] = a.f[(size_t)gy * a.f_pitch + gx];
        }
        return;
    }
    // the kept indices n = M .. N - M, unfolded: omega_n and w_n
    const int N = hd.N, M = hd.M, K = N - 2 * M + 1;
    const double scale = sqrt((double)N) * (double)pt.sigma_r;
    for (int k = tid; k < K; k += NT) {
        const int n = M + k;
        const double om = (double)(2 * n - N) / scale;
        float w;
        if (2 * n == N) w = hd.w0;
        else w = 0.5f * a.pairs[(2 * n > N ? n : N - n) - N / 2 - 1].W;
        tw_[3 * k] = (float)om;
        tw_[3 * k + 1] = (float)(om - (double)(float)om);
        tw_[3 * k + 2] = w;
    }
    for (int i = tid; i < G.ngz; i += NT) {
        const int t = i - 8;
        gz[i] = (t >= 0 && t <= 2 * R) ? a.taps[t] : 0.f;
    }
    for (int i = tid; i < (G.RHp - G.RH) * TW; i += NT)
        for (int q = 0; q < 4; ++q) hsm[q * hplane + (size_t)G.RH * TW + i] = 0.f;
    // centred f over the halo grown by one pixel (patch reach), clamped
    for (int r = warp; r < G.RH + 2; r += NW) {
        const int gy = min(max(gy0 + r - 1, 0), a.H - 1);
        for (int col = lane; col < EW; col += 32) {
            const int x = min(max(gx0 + col - 1, 0), a.W - 1);
            fext[r * EW + col] = __ldg(a.f + (size_t)gy * a.f_pitch + x) - a.c0;
        }
    }
    __syncthreads();
    for (int r = warp; r < G.RH; r += NW) {
        const int gy = gy0 + r;
        const bool rin = gy >= 0 && gy < a.H;
        for (int col = lane; col < G.RWp; col += 32) {
            const int x = gx0 + col;
            const bool in = rin && col < G.RW && x >= 0 && x < a.W;
            fsm[r * G.RWp + col] = in ? fext[(r + 1) * EW + col + 1] : 0.f;
        }
    }
    const float full = full_mass(a.taps, R);
    const float cmass = clipped_mass(a.taps, R, gx, a.W, full);
    float num[8], den[8], numc[8], denc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) num[i] = den[i] = numc[i] = denc[i] = 0.f;
    __syncthreads();

    long long total = 1;
    for (int i = 0; i < pt.p; ++i) total *= K;
    const long long half = (total + 1) / 2;
    for (long long t = 0; t < half; ++t) {
        // digits of the multi-index (base K, component 0 least significant)
        int dig[kMaxPatch];
        float Wnu = (2 * t + 1 == total) ? 1.f : 2.f;
        long long r_ = t;
        for (int i = 0; i < pt.p; ++i) {
            dig[i] = (int)(r_ % K);
            r_ /= K;
            Wnu *= tw_[3 * dig[i] + 2];
        }
        // (1) modulate: cos / sin of the patch phase at every in-image halo pixel
        for (int r = warp; r < G.RH; r += NW) {
            const int gy = gy0 + r;
            const bool rin = gy >= 0 && gy < a.H;
            for (int col = lane; col < G.RWp; col += 32) {
                const int x = gx0 + col;
                float c = 0.f, s = 0.f;
                if (rin && col < G.RW && x >= 0 && x < a.W) {
                    float hi = 0.f, lo = 0.f;
                    for (int i = 0; i < pt.p; ++i) {
                        const float v = fext[(r + 1 + pt.uy[i]) * EW + col + 1 + pt.ux[i]];
                        const float oh = tw_[3 * dig[i]], ol = tw_[3 * dig[i] + 1];
                        const float pr = __fmul_rn(oh, v);
                        const float e = fmaf(oh, v, -pr);          // exact error of pr
                        const float sh = __fadd_rn(hi, pr);         // two-sum of the heads
                        const float bp = __fsub_rn(sh, hi);
                        lo += (hi - (sh - bp)) + (pr - bp) + e + ol * v;
                        hi = sh;
                    }
                    const float q = rintf(__fmul_rn(hi, fir32::kInv2Pi));
                    float rr = fmaf(-q, fir32::k2PiHi, hi);
                    rr = fmaf(-q, fir32::k2PiLo, rr);
                    rr = __fadd_rn(rr, lo);
                    __sincosf(rr, &s, &c);
                }
                csm[r * G.RWp + col] = c;
                ssm[r * G.RWp + col] = s;
            }
        }
        __syncthreads();
        // (2) rows: planes (f c, f s, c, s)
        fir32::row_pass<TW, true>(G, fsm, nullptr, csm, ssm, gz, hsm, tid, NT);
        __syncthreads();
        // (3) columns, then demodulate with the output pixel's own phase
        {
            float acc[4][8];
            fir32::col_pass<TW>(G, hsm, gz, o, rb, acc);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int ry = rb * 8 + i + R;
                const float c = csm[ry * G.RWp + o + R], s = ssm[ry * G.RWp + o + R];
                comp_add(num[i], numc[i], Wnu * fmaf(c, acc[0][i], s * acc[1][i]));
                comp_add(den[i], denc[i], Wnu * fmaf(c, acc[2][i], s * acc[3][i]));
            }
        }
        __syncthreads();
    }

    if (gx < a.W) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gy = by + rb * 8 + i;
            if (gy >= a.H) continue;
            num[i] += numc[i];
            den[i] += denc[i];
            const float rmass = clipped_mass(a.taps, R, gy, a.H, full);
            float v;
            if (den[i] > kGuard * rmass * cmass) {
                v = __fdiv_rn(num[i], den[i]) + a.c0;
            } else {
                v = a.f[(size_t)gy * a.f_pitch + gx];
                atomicAdd(a.n_guarded, 1ull);
            }
            a.out[(size_t)gy * a.out_pitch + gx] = v;
        }
    }
}

template <int TH, int TW>
cudaError_t launch_nlm_tile(const FwdArgs& a, const NlmPatch& pt, int n_cap, cudaStream_t s)
{
    const size_t smem = nlm_smem_bytes(a.R, TH, TW, n_cap);
    cudaError_t e = cudaFuncSetAttribute(k_nlm32<TH, TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    k_nlm32<TH, TW><<<grid, TH * TW / 8, smem, s>>>(a, pt);
    return cudaGetLastError();
}

}  // namespace

size_t nlm_smem_bytes(int R, int th, int tw, int n_cap)
{
    const Geo G(R, th, tw);
    const size_t ext = (size_t)(G.RH + 2) * (G.RWp + 2);
    return sizeof(float) * (ext + G.floats(tw, 3) + 3 * ((size_t)n_cap + 1));
}

void nlm_tile(int R, int n_cap, int* th, int* tw)
{
    static const int shapes[][2] = {{64, 32}, {32, 32}, {16, 16}};
    for (auto& sh : shapes)
        if (nlm_smem_bytes(R, sh[0], sh[1], n_cap) <= 227 * 1024) {
            *th = sh[0];
            *tw = sh[1];
            return;
        }
    *th = *tw = 0;
}

cudaError_t launch_nlm32(const FwdArgs& a, const NlmPatch& pt, int n_cap, cudaStream_t s)
{
    if (pt.p < 1 || pt.p > kMaxPatch || a.set_tile) return cudaErrorInvalidValue;
    int th = 0, tw = 0;
    nlm_tile(a.R, n_cap, &th, &tw);
    if (th == 64 && tw == 32) return launch_nlm_tile<64, 32>(a, pt, n_cap, s);
    if (th == 32 && tw == 32) return launch_nlm_tile<32, 32>(a, pt, n_cap, s);
    if (th == 16 && tw == 16) return launch_nlm_tile<16, 16>(a, pt, n_cap, s);
    return cudaErrorInvalidValue;
}

}  // namespace bf
