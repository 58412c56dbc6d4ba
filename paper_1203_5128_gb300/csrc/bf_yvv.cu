// K3-yvv: SHIFTABLE-BF (Sec. 1.2) with a recursive Gaussian in step 2.
//
// Sec. 1.2 lets the Gaussian filtering of the modulated planes be done by an
// O(1) recursive filter.  This one is the third-order recursion of Young and
// van Vliet (Signal Processing 44, 1995): a causal pass and an anti-causal
// pass with the same poles, on the plane extended by zeros without limit,
// rows and then columns.  Its cost per sample does not depend on sigma_s.
//
// Form of the recursion.  The cascade (causal, then anti-causal) has the
// symmetric impulse response h[n] = sum_i c_i p_i^|n| over its three poles
// (one real, one complex pair), so the same filter is the sum of a causal
// part sum_{m>=0} h[m] x[n-m] and an anti-causal part sum_{m>=1} h[m] x[n+m],
// each a first-order section per pole:
//   causal       u_i[n] = p_i u_i[n-1] + x[n],   y+[n] = sum_i c_i u_i[n]
//   anti-causal  v_i[n] = p_i v_i[n+1] + x[n],   y-[n] = sum_i c_i p_i v_i[n+1]
// both starting from zero state at the ends of the line, which is exact for
// the zero extension (no margin).  First-order sections keep the FP32
// rounding small (the gain of one section is 1 / (1 - |p|)); the direct
// third-order form would amplify it by the whole filter's DC gain
// b0 / (b0 - b1 - b2 - b3), two orders of magnitude more at sigma_s = 8.
//
// Because the filtered planes are demodulated and summed linearly, the
// column pass never materialises its output: the down sweep adds the causal
// part's contribution to num and den, the up sweep the anti-causal part's.
//
// Kernels, per pass of C terms (C in {8, 16}; lanes = 32 / C lines x C
// terms, term k = pass * C + lane % C, the zero frequency as term F with
// omega = 0 and weight w0):
//   k_yvv_rows  one warp per 32 / C rows: planes f'c, f's, c, s of each term
//               (f' = f - value_range / 2), filtered along the row and written
//               once to P[y][x][term][4] (two sweeps, see below);
//   k_yvv_cols  one warp per 32 / C columns: down and up sweeps over P,
//               demodulation with the term's cos, sin at the output pixel, a
//               shuffle sum over the C terms, accumulated into (num, den);
//   k_yvv_final num / den + value_range / 2, with the denominator guard
//               against 1e-6 times the filter of the image's indicator
//               (separable: mass_y[y] mass_x[x]).
// The number of passes follows the plan's cap on N (the host never reads
// the device's N); passes beyond the set's terms return at once.  Each
// launch runs G = 32 / C passes side by side (grid.y); pass group g keeps
// its own (num, den) partial, and the final kernel adds the G partials in
// group order, so the result does not depend on scheduling.
#include <complex>
#include <math.h>

#include "bf_fir32.cuh"

namespace bf {

namespace {

constexpr int kWarpsPerCta = 4;

// Two planes' first-order sections side by side: lane x and lane y of
// each float2 are two planes, advanced together by packed multiply-adds
// (fma.rn.f32x2; each lane rounds like fmaf).  The planes are paired as
// (f'c, c) and (f's, s), so that the demodulation of one output forms
// (num, den) as a pair.
struct Sec2 {
    float2 a, re, im;     // real-pole state, complex-pole state
};

// u <- p u + x for the real pole and the complex pole.
__device__ __forceinline__ void sec_update(Sec2& s, float2 x, const YvvCoef2& k)
{
    s.a = __ffma2_rn(k.P0, s.a, x);
    const float2 re = __ffma2_rn(k.Pr, s.re, __ffma2_rn(k.nPi, s.im, x));
    const float2 im = __ffma2_rn(k.Pr, s.im, __fmul2_rn(k.Pi, s.re));
    s.re = re;
    s.im = im;
}

// c0 u_0 + 2 Re(c1 u_1): the causal output after the update.
__device__ __forceinline__ float2 sec_causal_out(const Sec2& s, const YvvCoef2& k)
{
    return __ffma2_rn(k.C0, s.a, __ffma2_rn(k.Cr, s.re, __fmul2_rn(k.nCi, s.im)));
}

// c0 p0 v_0 + 2 Re(c1 p1 v_1): the anti-causal output, before the update.
__device__ __forceinline__ float2 sec_anti_out(const Sec2& s, const YvvCoef2& k)
{
    return __ffma2_rn(k.D0, s.a, __ffma2_rn(k.Dr, s.re, __fmul2_rn(k.nDi, s.im)));
}

__device__ __forceinline__ void term_of(const YvvArgs& a, const SetHdr& hd, int k, float& om_hi,
                                        float& om_lo, float& Wk)
{
    om_hi = om_lo = Wk = 0.f;
    if (k < hd.F) {
        const Pair p = a.pairs[k];
        om_hi = p.om_hi;
        om_lo = p.om_lo;
        Wk = p.W;
    } else if (k == hd.F && hd.z) {
        Wk = hd.w0;        // zero frequency: cos = 1, sin = 0
    }
}

// The plane pairs (v c, c) and (v s, s) of a sample.
__device__ __forceinline__ void planes_at(float v, float om_hi, float om_lo, float2 (&in)[2])
{
    float c, s;
    fir32::phase_cs(v, om_hi, om_lo, c, s);
    in[0] = make_float2(v * c, c);
    in[1] = make_float2(v * s, s);
}

// Row kernel in two sweeps so that each row-filtered sample is written once:
//   A (right to left): the anti-causal states only; the state entering each
//     chunk of kRowChunk samples from the right, v[x0 + kRowChunk], is saved
//     (12 floats per term; the last chunk's is zero);
//   B (left to right, chunk by chunk): the chunk's planes in registers, the
//     anti-causal part from the saved state (right to left within the chunk),
//     then the causal part, and y+ + y- stored once.
constexpr int kRowChunk = 8;

template <int C>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_yvv_rows(YvvArgs a, int launch)
{
    constexpr int LPW = 32 / C;                    // lines per warp
    constexpr int B = kRowChunk;
    const int GC = a.G * C;                        // term columns per launch
    const int g = blockIdx.y;                      // pass group of this CTA
    const int pass = launch * a.G + g;
    const int lane = threadIdx.x & 31;
    const int slot = lane % C;
    const int y = (blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5)) * LPW + lane / C;
    const SetHdr hd = a.hdr[0];
    const int nterms = hd.F < 0 ? 0 : hd.F + hd.z;
    if (pass * C >= nterms || y >= a.H) return;
    const int k = pass * C + slot;
    const bool act = k < nterms;
    float om_hi, om_lo, Wk;
    term_of(a, hd, k, om_hi, om_lo, Wk);
    const YvvCoef2& cf = a.coef2;
    const int W = a.W;
    const int nch = (W + B - 1) / B;
    const int col = g * C + slot;
    const float* frow = a.f + (size_t)y * a.f_pitch;
    float4* P = a.P + (size_t)y * W * GC + col;            // (y, x, col) at P[x * GC]
    float4* S = a.S + (size_t)y * nch * 3 * GC + col;      // (y, chunk, t, col) at S[(j * 3 + t) * GC]

    // sweep A: anti-causal states at the chunk boundaries (the next chunk's
    // f is fetched while this one is processed)
    const float2 z2 = make_float2(0.f, 0.f);
    Sec2 st[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) st[q] = Sec2{z2, z2, z2};
    float fn[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const int x = (nch - 1) * B + i;
        fn[i] = x < W ? __ldg(frow + x) : 0.f;
    }
    for (int j = nch - 1; j >= 0; --j) {
        if (act) {
            float4* d = S + (size_t)j * 3 * GC;
            d[0] = make_float4(st[0].a.x, st[0].a.y, st[0].re.x, st[0].re.y);
            d[GC] = make_float4(st[0].im.x, st[0].im.y, st[1].a.x, st[1].a.y);
            d[2 * GC] = make_float4(st[1].re.x, st[1].re.y, st[1].im.x, st[1].im.y);
        }
        const int x0 = j * B;
        float fv[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            fv[i] = fn[i];
            fn[i] = j > 0 ? __ldg(frow + x0 - B + i) : 0.f;
        }
#pragma unroll
        for (int i = B - 1; i >= 0; --i) {
            if (x0 + i >= W) continue;
            float2 in[2];
            planes_at(fv[i] - a.c0, om_hi, om_lo, in);
#pragma unroll
            for (int q = 0; q < 2; ++q) sec_update(st[q], in[q], cf);
        }
    }
    // sweep B: both parts per chunk, one store per sample (the next chunk's
    // saved state and f are fetched while this one is processed)
    Sec2 cs[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) cs[q] = Sec2{z2, z2, z2};
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 n0 = act ? S[0] : z4, n1 = act ? S[GC] : z4, n2 = act ? S[2 * GC] : z4;
#pragma unroll
    for (int i = 0; i < B; ++i) fn[i] = i < W ? __ldg(frow + i) : 0.f;
    for (int j = 0; j < nch; ++j) {
        const int x0 = j * B;
        Sec2 vs[2];
        vs[0] = Sec2{make_float2(n0.x, n0.y), make_float2(n0.z, n0.w), make_float2(n1.x, n1.y)};
        vs[1] = Sec2{make_float2(n1.z, n1.w), make_float2(n2.x, n2.y), make_float2(n2.z, n2.w)};
        float fv[B];
#pragma unroll
        for (int i = 0; i < B; ++i) fv[i] = fn[i];
        if (j + 1 < nch) {
            const float4* d = S + (size_t)(j + 1) * 3 * GC;
            n0 = act ? d[0] : z4;
            n1 = act ? d[GC] : z4;
            n2 = act ? d[2 * GC] : z4;
#pragma unroll
            for (int i = 0; i < B; ++i) fn[i] = x0 + B + i < W ? __ldg(frow + x0 + B + i) : 0.f;
        }
        float2 in[B][2], ym[B][2];
#pragma unroll
        for (int i = 0; i < B; ++i) planes_at(x0 + i < W ? fv[i] - a.c0 : 0.f, om_hi, om_lo, in[i]);
#pragma unroll
        for (int i = B - 1; i >= 0; --i) {
            if (x0 + i >= W) continue;            // past the row: the state stays v[W] = 0
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                ym[i][q] = sec_anti_out(vs[q], cf);
                sec_update(vs[q], in[i][q], cf);
            }
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            if (x0 + i >= W) break;
            float2 o[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                sec_update(cs[q], in[i][q], cf);
                o[q] = __fadd2_rn(sec_causal_out(cs[q], cf), ym[i][q]);
            }
            if (act) P[(size_t)(x0 + i) * GC] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        }
    }
}

template <int C>
__device__ __forceinline__ void reduce_terms(float& nu, float& de)
{
#pragma unroll
    for (int o = C / 2; o >= 1; o >>= 1) {
        nu += __shfl_xor_sync(0xffffffffu, nu, o);
        de += __shfl_xor_sync(0xffffffffu, de, o);
    }
}

// cp.async of 16, 8 or 4 bytes into shared memory, zero-filled when !pred
// (nothing is read then; src must still be a valid address).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "r"(pred ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool pred)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "r"(pred ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool pred)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "r"(pred ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

constexpr int kColChunk = 8;      // rows per chunk of the column sweeps

// Shared memory of one warp of the column kernel: two stages of a chunk
// (planes of 32 lanes, f and the (num, den) partials of the warp's columns).
struct ColStage {
    float4 P[kColChunk][32];
    float f[4][kColChunk];
    float2 nd[4][kColChunk];
};

template <int C>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_yvv_cols(YvvArgs a, int launch)
{
    constexpr int LPW = 32 / C;
    constexpr int B = kColChunk;
    __shared__ ColStage stage_sm[kWarpsPerCta][2];
    const int GC = a.G * C;
    const int g = blockIdx.y;
    const int pass = launch * a.G + g;
    const int lane = threadIdx.x & 31;
    const int slot = lane % C;
    const int wl = threadIdx.x >> 5;
    const int x0w = (blockIdx.x * kWarpsPerCta + wl) * LPW;     // first column of the warp
    const int x = x0w + lane / C;
    const SetHdr hd = a.hdr[0];
    const int nterms = hd.F < 0 ? 0 : hd.F + hd.z;
    if (pass * C >= nterms) {                     // uniform over the CTA
        // a group without terms in the first launch still owns a partial
        // that the final kernel sums: zero it
        if (launch == 0 && x < a.W && slot == 0) {
            float2* ND = a.nd + (size_t)g * a.H * a.W + x;
            for (int y = 0; y < a.H; ++y) ND[(size_t)y * a.W] = make_float2(0.f, 0.f);
        }
        return;
    }
    // lanes past the last column stay for the shuffles
    if (x0w >= a.W) return;                       // whole warp out
    const bool xin = x < a.W;
    const int k = pass * C + slot;
    const bool act = xin && k < nterms;
    float om_hi, om_lo, Wk;
    term_of(a, hd, k, om_hi, om_lo, Wk);
    if (!act) Wk = 0.f;
    const YvvCoef2& cf = a.coef2;
    const int H = a.H, W = a.W;
    const int xc = xin ? x : 0;
    const float4* P = a.P + (size_t)xc * GC + g * C + slot;   // (y, x, col) at P[y * W * GC]
    const size_t pstride = (size_t)W * GC;
    float2* ND = a.nd + (size_t)g * H * W + xc;     // this group's partial (num, den)
    const bool writer = xin && slot == 0;
    const bool first = launch == 0;
    ColStage* stg = stage_sm[wl];
    // the (row j, column sub) of f and (num, den) this lane fetches for a chunk
    const int fj = lane % B, fsub = lane / B;
    const int fx = x0w + fsub;
    const bool fcol_ok = fsub < LPW && fx < W;
    const float* fsrc = a.f + (fcol_ok ? fx : 0);
    float2* ndsrc = a.nd + (size_t)g * H * W + (fcol_ok ? fx : 0);

    // chunk c of a sweep covers rows y(c, j) = down ? cB + j : H - 1 - (cB + j)
    auto fetch = [&](int c, bool down, bool need_nd) {
        ColStage& st = stg[c & 1];
#pragma unroll
        for (int jj = 0; jj < B; ++jj) {
            const int r = c * B + jj;
            const int y = down ? r : H - 1 - r;
            const bool ok = act && r < H;
            cp_async16(&st.P[jj][lane], ok ? (const void*)(P + (size_t)y * pstride) : (const void*)a.P, ok);
        }
        {
            const int r = c * B + fj;
            const int y = down ? r : H - 1 - r;
            const bool ok = fcol_ok && r < H;
            if (fsub < 4) {
                cp_async4(&st.f[fsub][fj], ok ? (const void*)(fsrc + (size_t)y * a.f_pitch) : (const void*)a.f, ok);
                cp_async8(&st.nd[fsub][fj], (ok && need_nd) ? (const void*)(ndsrc + (size_t)y * W) : (const void*)a.nd,
                          ok && need_nd);
            }
        }
        cp_async_commit();
    };
    const int nchunk = (H + B - 1) / B;
    const int sub = lane / C;

    const float2 z2 = make_float2(0.f, 0.f);
    const float2 W2 = make_float2(Wk, Wk);
    Sec2 st[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) st[q] = Sec2{z2, z2, z2};
    // down sweep: causal part
    fetch(0, true, !first);
    for (int c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) fetch(c + 1, true, !first);
        else cp_async_commit();                   // empty group keeps the count
        cp_async_wait1();
        __syncwarp();
        const ColStage& sc = stg[c & 1];
        float2 acc[B];
#pragma unroll
        for (int jj = 0; jj < B; ++jj) {
            const float4 cur = sc.P[jj][lane];
            sec_update(st[0], make_float2(cur.x, cur.y), cf);
            sec_update(st[1], make_float2(cur.z, cur.w), cf);
            float cc, ss;
            fir32::phase_cs(sc.f[sub][jj] - a.c0, om_hi, om_lo, cc, ss);
            // (num, den) = Wk (c (oA, oC) + s (oB, oD))
            const float2 nd = __fmul2_rn(W2, __ffma2_rn(make_float2(cc, cc), sec_causal_out(st[0], cf),
                                                        __fmul2_rn(make_float2(ss, ss),
                                                                   sec_causal_out(st[1], cf))));
            float nu = nd.x, de = nd.y;
            reduce_terms<C>(nu, de);
            acc[jj] = first ? make_float2(nu, de)
                            : make_float2(sc.nd[sub][jj].x + nu, sc.nd[sub][jj].y + de);
        }
        if (writer) {
#pragma unroll
            for (int jj = 0; jj < B; ++jj)
                if (c * B + jj < H) ND[(size_t)(c * B + jj) * W] = acc[jj];
        }
        __syncwarp();                             // stage c & 1 is refilled next
    }
    // up sweep: anti-causal part (rows H-1 down to 0); its (num, den) reads
    // see the down sweep's stores (same thread wrote them, or the writer of
    // the same column before this warp-wide point)
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 2; ++q) st[q] = Sec2{z2, z2, z2};
    fetch(0, false, true);
    for (int c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) fetch(c + 1, false, true);
        else cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        const ColStage& sc = stg[c & 1];
        float2 acc[B];
#pragma unroll
        for (int jj = 0; jj < B; ++jj) {
            const float4 cur = sc.P[jj][lane];
            const float2 oAC = sec_anti_out(st[0], cf), oBD = sec_anti_out(st[1], cf);
            sec_update(st[0], make_float2(cur.x, cur.y), cf);
            sec_update(st[1], make_float2(cur.z, cur.w), cf);
            float cc, ss;
            fir32::phase_cs(sc.f[sub][jj] - a.c0, om_hi, om_lo, cc, ss);
            const float2 nd = __fmul2_rn(W2, __ffma2_rn(make_float2(cc, cc), oAC,
                                                        __fmul2_rn(make_float2(ss, ss), oBD)));
            float nu = nd.x, de = nd.y;
            reduce_terms<C>(nu, de);
            acc[jj] = make_float2(sc.nd[sub][jj].x + nu, sc.nd[sub][jj].y + de);
        }
        if (writer) {
#pragma unroll
            for (int jj = 0; jj < B; ++jj) {
                const int y = H - 1 - (c * B + jj);
                if (y >= 0) ND[(size_t)y * W] = acc[jj];
            }
        }
        __syncwarp();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__global__ void k_yvv_final(YvvArgs a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.W) return;
    const SetHdr hd = a.hdr[0];
    for (int y = blockIdx.y; y < a.H; y += gridDim.y) {
        const float fv = a.f[(size_t)y * a.f_pitch + x];
        float v;
        if (hd.F < 0) {
            v = fv;                                  // order above the cap: pass through
        } else {
            // the groups' partial sums, in group order
            const size_t hw = (size_t)a.H * a.W;
            float2 nd = make_float2(0.f, 0.f);
            for (int g = 0; g < a.n_nd; ++g) {
                const float2 t = a.nd[g * hw + (size_t)y * a.W + x];
                nd.x += t.x;
                nd.y += t.y;
            }
            if (nd.y > kGuard * (a.mass_y[y] * a.mass_x[x])) {
                v = __fdiv_rn(nd.x, nd.y) + a.c0;
            } else {
                v = fv;
                atomicAdd(a.n_guarded, 1ull);
            }
        }
        a.out[(size_t)y * a.out_pitch + x] = v;
    }
}

}  // namespace

// ---- plan-time design (host, double) ---------------------------------------

bool yvv_design(double sigma, YvvCoef* out, double* poles_c /* [6]: p0, Re p1, Im p1, c0, Re c1, Im c1 */)
{
    if (!(sigma >= 0.5) || !isfinite(sigma)) return false;
    // published coefficients of the recursion (Young and van Vliet 1995)
    const double q = sigma >= 2.5 ? 0.98711 * sigma - 0.96330
                                  : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * sigma);
    const double b0 = 1.57825 + q * (2.44413 + q * (1.4281 + q * 0.422205));
    const double b1 = q * (2.44413 + q * (2.85619 + q * 1.26661));
    const double b2 = -q * q * (1.4281 + q * 1.26661);
    const double b3 = 0.422205 * q * q * q;
    const double a1 = b1 / b0, a2 = b2 / b0, a3 = b3 / b0;
    const double B = 1.0 - (a1 + a2 + a3);
    // poles: roots of z^3 - a1 z^2 - a2 z - a3; P(0) = -a3 < 0 < P(1) = B,
    // so one real root lies in (0, 1) (bisection to the last bit); the other
    // two are the roots of the deflated quadratic z^2 + bq z + cq.
    auto P = [&](double z) { return ((z - a1) * z - a2) * z - a3; };
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        (P(mid) < 0.0 ? lo : hi) = mid;
    }
    const double r = 0.5 * (lo + hi);
    const double bq = r - a1, cq = a3 / r;
    const double disc = 4.0 * cq - bq * bq;
    if (!(disc > 0.0)) return false;          // the published design has a complex pair
    using cd = std::complex<double>;
    const cd p[3] = {cd(r, 0.0), cd(-0.5 * bq, 0.5 * sqrt(disc)), cd(-0.5 * bq, -0.5 * sqrt(disc))};
    // 1 / prod_j (1 - p_j / z) = sum_i al_i / (1 - p_i / z), al_i = p_i^2 / prod_{j != i} (p_i - p_j)
    cd al[3];
    for (int i = 0; i < 3; ++i) {
        cd d(1.0, 0.0);
        for (int j = 0; j < 3; ++j)
            if (j != i) d *= p[i] - p[j];
        al[i] = p[i] * p[i] / d;
    }
    // h[n] = B^2 sum_m g[m + n] g[m], g[m] = sum_i al_i p_i^m, gives
    // h[n] = sum_i c_i p_i^n with c_i = B^2 al_i sum_j al_j / (1 - p_i p_j)
    cd c[3];
    for (int i = 0; i < 3; ++i) {
        cd sacc(0.0, 0.0);
        for (int j = 0; j < 3; ++j) sacc += al[j] / (1.0 - p[i] * p[j]);
        c[i] = B * B * al[i] * sacc;
    }
    const cd d1 = c[1] * p[1];
    out->P0 = (float)r;
    out->Pr = (float)p[1].real();
    out->Pi = (float)p[1].imag();
    out->C0 = (float)c[0].real();
    out->Cr = (float)(2.0 * c[1].real());
    out->Ci = (float)(2.0 * c[1].imag());
    out->D0 = (float)(c[0].real() * r);
    out->Dr = (float)(2.0 * d1.real());
    out->Di = (float)(2.0 * d1.imag());
    if (poles_c) {
        poles_c[0] = r;
        poles_c[1] = p[1].real();
        poles_c[2] = p[1].imag();
        poles_c[3] = c[0].real();
        poles_c[4] = c[1].real();
        poles_c[5] = c[1].imag();
    }
    return true;
}

// Filter of the indicator of [0, n) at each of its n samples, in double:
// the causal and anti-causal first-order sections of yvv_design run on ones.
void yvv_line_mass(double sigma, int n, float* mass)
{
    double pc[6];
    YvvCoef k;
    if (!yvv_design(sigma, &k, pc)) return;
    using cd = std::complex<double>;
    const double p0 = pc[0];
    const cd p1(pc[1], pc[2]);
    const double c0 = pc[3];
    const cd c1(pc[4], pc[5]);
    double u0 = 0.0;
    cd u1(0.0, 0.0);
    for (int i = 0; i < n; ++i) {
        u0 = p0 * u0 + 1.0;
        u1 = p1 * u1 + 1.0;
        mass[i] = (float)(c0 * u0 + 2.0 * (c1 * u1).real());
    }
    double v0 = 0.0;
    cd v1(0.0, 0.0);
    for (int i = n - 1; i >= 0; --i) {
        mass[i] = (float)((double)mass[i] + c0 * p0 * v0 + 2.0 * (c1 * p1 * v1).real());
        v0 = p0 * v0 + 1.0;
        v1 = p1 * v1 + 1.0;
    }
}

// 8 terms per pass for small orders, else 16: at most 15 idle lanes in the
// last pass whatever the device's N (32 would waste up to 31).  32 / C
// passes run side by side in one launch (grid.y), so that every launch has
// one warp per line: the line recursions are sequential and need the warps.
int yvv_terms_per_pass(int n_terms_cap) { return n_terms_cap <= 8 ? 8 : 16; }

cudaError_t launch_yvv(const YvvArgs& a0, int C, int n_passes, cudaStream_t s)
{
    YvvArgs a = a0;
    const int G = a.G;
    const int n_launch = (n_passes + G - 1) / G;
    a.n_nd = G;                                   // every group's partial is written at launch 0
    const int lines_per_cta = kWarpsPerCta * (32 / C);
    const dim3 block(32 * kWarpsPerCta);
    const dim3 grow((a.H + lines_per_cta - 1) / lines_per_cta, G);
    const dim3 gcol((a.W + lines_per_cta - 1) / lines_per_cta, G);
    for (int l = 0; l < n_launch; ++l) {
        switch (C) {
        case 8:
            k_yvv_rows<8><<<grow, block, 0, s>>>(a, l);
            k_yvv_cols<8><<<gcol, block, 0, s>>>(a, l);
            break;
        case 16:
            k_yvv_rows<16><<<grow, block, 0, s>>>(a, l);
            k_yvv_cols<16><<<gcol, block, 0, s>>>(a, l);
            break;
        default:
            return cudaErrorInvalidValue;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_yvv_final<<<dim3((a.W + 255) / 256, a.H < 65535 ? a.H : 65535), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bf
