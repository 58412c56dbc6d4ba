// K5: hand-written adjoint of the shiftable filter (FP32 planes, FIR).
//
// Not in the paper; derived from eqs. (f1)-(f2).  With P = sum_k W_k Re(...)
// the numerator and Q the denominator of SHIFTABLE-BF at x, out = P / Q,
// and L = sum_x u(x) out(x), write a = u / Q and b = -u P / Q^2 = -a (out - c0)
// (centred image f' = f - c0).  With c, s = cos, sin(w f'), G the clipped
// Gaussian filter (self-adjoint: the window is symmetric and clipping is the
// same on both sides) and A = G(f' c), B = G(f' s), C = G(c), D = G(s):
//
//   dL/df(z) = sum_k W_k [ c G(ac) + s G(as) - w f' (s G(ac) - c G(as))
//                          - w (s G(bc) - c G(bs))
//                          + w a (c B - s A) + w b (c D - s C) ](z)
//
// (the first line is the derivative through the neighbour f(y), the last
// through the centre f(x); every term is even in w, so the pair n, N-n folds
// into W_k = 2 w_n like the forward; the zero frequency gives w0 G(a)).
// T, N, M and the denominator guard are held at the forward's values; at a
// guarded pixel out = f, so a = b = 0 there and dL/df gets u.
//
// GB300 form: as the forward K3 -- one CTA per output tile, halo staged in
// shared memory once, per pair the four forward planes and then the four
// adjoint planes go through the same register-blocked row and column FIR,
// and the combination is accumulated in registers.  The forward values out
// and den over the halo come from a forward pass run just before (bf_backward).
// For Rp = 4 ceil(R/4) <= 20 the 64 x 32 tile takes the packed-pair form of
// the tall forward (k_bwd32x): (cos, sin) interleaved, the pairs (f'c, f's),
// (c, s), (ac, as), (bc, bs) filtered with fma.rn.f32x2 and constant-bank
// taps; larger radii keep the scalar form (k_bwd32).
#include <math.h>

#include "bf_fir32.cuh"

namespace bf {
namespace {

using fir32::Geo;
using fir32::phase_cs;

template <int TH, int TW>
__global__ void __launch_bounds__(TH * TW / 8, 1) k_bwd32(BwdArgs a)
{
    constexpr int NT = TH * TW / 8;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) float sm[];
    const Geo G(a.R, TH, TW);
    const int R = a.R;
    const size_t rsz = (size_t)G.RH * G.RWp;
    float* fsm = sm;                      // centred f
    float* csm = fsm + rsz;               // cos
    float* ssm = csm + rsz;               // sin
    float* asm_ = ssm + rsz;              // a = u / den
    float* bsm = asm_ + rsz;              // b = -a (out - c0)
    float* hsm = bsm + rsz;               // 4 x RHp x TW row-filtered planes
    float* gz = hsm + 4 * (size_t)G.RHp * TW;
    float* rmass = gz + G.ngz;            // clipped Gaussian mass of each halo row
    float* cmass = rmass + G.RH;          // ... and column

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int by = blockIdx.y * TH, bx = blockIdx.x * TW;
    const int gy0 = by - R, gx0 = bx - R;
    const int set = a.set_tile ? (by / a.set_tile) * a.sets_x + (bx / a.set_tile) : 0;
    const SetHdr hd = a.hdr[set];
    const int o = tid % TW, rb = tid / TW;
    const int gx = bx + o;

    for (int i = tid; i < G.ngz; i += NT) {
        const int t = i - 8;
        gz[i] = (t >= 0 && t <= 2 * R) ? a.taps[t] : 0.f;
    }
    // same summation order as the forward's guard
    for (int r = tid; r < G.RH; r += NT) {
        const int gy = gy0 + r;
        float m = 0.f;
        for (int t = -R; t <= R; ++t)
            if (gy + t >= 0 && gy + t < a.H) m += a.taps[t + R];
        rmass[r] = m;
    }
    for (int c = tid; c < G.RW; c += NT) {
        const int x = gx0 + c;
        float m = 0.f;
        for (int t = -R; t <= R; ++t)
            if (x + t >= 0 && x + t < a.W) m += a.taps[t + R];
        cmass[c] = m;
    }
    for (int i = tid; i < (G.RHp - G.RH) * TW; i += NT)
        for (int q = 0; q < 4; ++q) hsm[q * (size_t)G.RHp * TW + (size_t)G.RH * TW + i] = 0.f;
    __syncthreads();

    // stage f' over the halo (0 outside the image and in the padding)
    for (int r = warp; r < G.RH; r += NW) {
        const int gy = gy0 + r;
        const bool rin = gy >= 0 && gy < a.H;
        for (int col = lane; col < G.RWp; col += 32) {
            const int x = gx0 + col;
            float fv = 0.f;
            if (rin && col < G.RW && x >= 0 && x < a.W)
                fv = __ldg(a.f + (size_t)gy * a.pitch + x) - a.c0;
            fsm[r * G.RWp + col] = fv;
        }
    }

    float grad[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) grad[i] = 0.f;

    // The neighbour terms of output x use x's own kernel: loop over the
    // T-tiles that meet the halo, with a and b restricted to each (one pass
    // when T is global or fixed).  The centre terms belong to this tile's set.
    int ty0 = 0, ty1 = 0, tx0 = 0, tx1 = 0;
    if (a.set_tile) {
        ty0 = max(gy0, 0) / a.set_tile;
        ty1 = min(gy0 + G.RH - 1, a.H - 1) / a.set_tile;
        tx0 = max(gx0, 0) / a.set_tile;
        tx1 = min(gx0 + G.RW - 1, a.W - 1) / a.set_tile;
    }
    for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
        const int tset = a.set_tile ? ty * a.sets_x + tx : 0;
        const bool own = tset == set;
        const SetHdr th = a.hdr[tset];
        // rectangle of outputs that use this set
        int ylo = 0, yhi = a.H, xlo = 0, xhi = a.W;
        if (a.set_tile) {
            ylo = ty * a.set_tile;
            yhi = min(ylo + a.set_tile, a.H);
            xlo = tx * a.set_tile;
            xhi = min(xlo + a.set_tile, a.W);
        }
        __syncthreads();
        // a = u / den, b = -a (out - c0) at the outputs of this set (0 where
        // the guard fired, outside the set and outside the image)
        for (int r = warp; r < G.RH; r += NW) {
            const int gy = gy0 + r;
            const bool rin = gy >= ylo && gy < yhi;
            for (int col = lane; col < G.RWp; col += 32) {
                const int x = gx0 + col;
                float av = 0.f, bv = 0.f;
                if (rin && col < G.RW && x >= xlo && x < xhi && th.F >= 0) {
                    const size_t k = (size_t)gy * a.pitch + x, ks = (size_t)gy * a.spitch + x;
                    const float d = a.den[ks];
                    if (d > kGuard * rmass[r] * cmass[col]) {
                        av = __fdiv_rn(__ldg(a.u + k), d);
                        bv = -av * (a.out[ks] - a.c0);
                    }
                }
                asm_[r * G.RWp + col] = av;
                bsm[r * G.RWp + col] = bv;
            }
        }
        __syncthreads();
        if (th.F < 0) continue;      // outputs of that set are copies of f: no neighbour terms

        const Pair* pr = a.pairs + (size_t)tset * a.cap_pairs;
        const int K = th.F + th.z;
        for (int k = 0; k < K; ++k) {
            float om_hi = 0.f, om_lo = 0.f, Wk = th.w0;
            if (k < th.F) {
                const Pair p = pr[k];
                om_hi = p.om_hi;
                om_lo = p.om_lo;
                Wk = p.W;
            }
            for (int r = warp; r < G.RH; r += NW) {
                const int gy = gy0 + r;
                const bool rin = gy >= 0 && gy < a.H;
                for (int col = lane; col < G.RWp; col += 32) {
                    const int x = gx0 + col;
                    float c = 0.f, s = 0.f;
                    if (rin && col < G.RW && x >= 0 && x < a.W)
                        phase_cs(fsm[r * G.RWp + col], om_hi, om_lo, c, s);
                    csm[r * G.RWp + col] = c;
                    ssm[r * G.RWp + col] = s;
                }
            }
            __syncthreads();
            // forward planes A, B, C, D at my outputs (centre terms, own set only)
            float accF[4][8];
            if (own) {
                fir32::row_pass<TW, true>(G, fsm, nullptr, csm, ssm, gz, hsm, tid, NT);
                __syncthreads();
                fir32::col_pass<TW>(G, hsm, gz, o, rb, accF);
                __syncthreads();
            }
            // adjoint planes: G(ac), G(as), G(bc), G(bs) at my outputs
            fir32::row_pass<TW, false>(G, asm_, bsm, csm, ssm, gz, hsm, tid, NT);
            __syncthreads();
            float accA[4][8];
            fir32::col_pass<TW>(G, hsm, gz, o, rb, accA);
            const float w = om_hi;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int zi = (rb * 8 + i + R) * G.RWp + o + R;
                const float c = csm[zi], s = ssm[zi], fz = fsm[zi];
                const float Gac = accA[0][i], Gas = accA[1][i], Gbc = accA[2][i], Gbs = accA[3][i];
                float v = fmaf(c, Gac, s * Gas);
                v = fmaf(-w * fz, fmaf(s, Gac, -c * Gas), v);
                v = fmaf(-w, fmaf(s, Gbc, -c * Gbs), v);
                if (own) {
                    const float az = asm_[zi], bz = bsm[zi];
                    v = fmaf(w * az, fmaf(c, accF[1][i], -s * accF[0][i]), v);
                    v = fmaf(w * bz, fmaf(c, accF[3][i], -s * accF[2][i]), v);
                }
                grad[i] = fmaf(Wk, v, grad[i]);
            }
            __syncthreads();
        }
    }

    if (gx < a.W) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gy = by + rb * 8 + i;
            if (gy >= a.H) continue;
            const int r = rb * 8 + i + R;
            const size_t k = (size_t)gy * a.pitch + gx;
            float g = grad[i];
            // out = f where the guard fired or the set passed the image through
            if (hd.F < 0 || !(a.den[(size_t)gy * a.spitch + gx] > kGuard * rmass[r] * cmass[o + R]))
                g += __ldg(a.u + k);
            a.grad[k] = g;
        }
    }
}

// Packed-pair form: 64 x 32 outputs, 256 threads (8 outputs of one column
// each), Rp = 4 (NCH - 1).  Shared memory: (cos, sin) RH x CSp float2; f', a,
// b RH x FP floats; two row-filtered pair planes RH x 32 float2; the clipped
// Gaussian mass of each halo row and column.
template <int TH, int NCH>
struct BwdGeo {
    static constexpr int TW = 32;
    static constexpr int Rp = 4 * (NCH - 1);
    static constexpr int RH = TH + 2 * Rp;
    static constexpr int RW = TW + 2 * Rp;
    static constexpr int CSp = RW + 2;
    static constexpr int FP = RW + 4;
    static constexpr size_t cs_bytes = (size_t)RH * CSp * 8;
    static constexpr size_t fz_bytes = (size_t)RH * FP * 4;
    static constexpr size_t hz_bytes = (size_t)RH * TW * 8;
    static constexpr size_t bytes = cs_bytes + 3 * fz_bytes + 2 * hz_bytes + 4 * (size_t)(RH + RW);
};

template <int TH, int NCH>
__global__ void __launch_bounds__(TH * 4, 1)
k_bwd32x(BwdArgs a, const __grid_constant__ fir32::Taps2 tp2)
{
    using G = BwdGeo<TH, NCH>;
    constexpr int TW = G::TW, NT = TH * TW / 8, Rp = G::Rp;
    extern __shared__ __align__(16) char smc[];
    float2* cs = (float2*)smc;
    float* fz = (float*)(smc + G::cs_bytes);
    float* az = fz + G::RH * G::FP;
    float* bz = az + G::RH * G::FP;
    float2* hz1 = (float2*)(bz + G::RH * G::FP);
    float2* hz2 = hz1 + G::RH * TW;
    float* rmass = (float*)(hz2 + G::RH * TW);
    float* cmass = rmass + G::RH;

    const int R = a.R;
    const int tid = threadIdx.x;
    const int by = blockIdx.y * TH, bx = blockIdx.x * TW;
    const int gy0 = by - Rp, gx0 = bx - Rp;
    const int set = a.set_tile ? (by / a.set_tile) * a.sets_x + (bx / a.set_tile) : 0;
    const SetHdr hd = a.hdr[set];
    const int o = tid % TW, rb = tid / TW;
    const int gx = bx + o;

    // same summation order as the forward's guard
    for (int r = tid; r < G::RH; r += NT) {
        const int gy = gy0 + r;
        float m = 0.f;
        for (int t = -R; t <= R; ++t)
            if (gy + t >= 0 && gy + t < a.H) m += a.taps[t + R];
        rmass[r] = m;
    }
    for (int c = tid; c < G::RW; c += NT) {
        const int x = gx0 + c;
        float m = 0.f;
        for (int t = -R; t <= R; ++t)
            if (x + t >= 0 && x + t < a.W) m += a.taps[t + R];
        cmass[c] = m;
    }
    // f' over the halo (0 outside the image)
    for (int e = tid; e < G::RH * G::RW; e += NT) {
        const int r = e / G::RW, col = e - r * G::RW;
        const int gy = gy0 + r, x = gx0 + col;
        float fv = 0.f;
        if (gy >= 0 && gy < a.H && x >= 0 && x < a.W)
            fv = __ldg(a.f + (size_t)gy * a.pitch + x) - a.c0;
        fz[r * G::FP + col] = fv;
    }
    using PS = fir32::PhaseSweep<G, NT>;
    const PS ps(tid, gy0, gx0, a.W);

    float grad[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) grad[i] = 0.f;

    // The neighbour terms of output x use x's own kernel: loop over the
    // T-tiles that meet the halo, with a and b restricted to each (one pass
    // when T is global or fixed).  The centre terms belong to this tile's set.
    int ty0 = 0, ty1 = 0, tx0 = 0, tx1 = 0;
    if (a.set_tile) {
        ty0 = max(gy0, 0) / a.set_tile;
        ty1 = min(gy0 + G::RH - 1, a.H - 1) / a.set_tile;
        tx0 = max(gx0, 0) / a.set_tile;
        tx1 = min(gx0 + G::RW - 1, a.W - 1) / a.set_tile;
    }
    for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
        const int tset = a.set_tile ? ty * a.sets_x + tx : 0;
        const bool own = tset == set;
        const SetHdr th = a.hdr[tset];
        int ylo = 0, yhi = a.H, xlo = 0, xhi = a.W;
        if (a.set_tile) {
            ylo = ty * a.set_tile;
            yhi = min(ylo + a.set_tile, a.H);
            xlo = tx * a.set_tile;
            xhi = min(xlo + a.set_tile, a.W);
        }
        __syncthreads();
        // a = u / den, b = -a (out - c0) at the outputs of this set (0 where
        // the guard fired, outside the set and outside the image)
        for (int e = tid; e < G::RH * G::RW; e += NT) {
            const int r = e / G::RW, col = e - r * G::RW;
            const int gy = gy0 + r, x = gx0 + col;
            float av = 0.f, bv = 0.f;
            if (gy >= ylo && gy < yhi && x >= xlo && x < xhi && th.F >= 0) {
                const size_t k = (size_t)gy * a.pitch + x, ks = (size_t)gy * a.spitch + x;
                const float d = a.den[ks];
                if (d > kGuard * rmass[r] * cmass[col]) {
                    av = __fdiv_rn(__ldg(a.u + k), d);
                    bv = -av * (a.out[ks] - a.c0);
                }
            }
            az[r * G::FP + col] = av;
            bz[r * G::FP + col] = bv;
        }
        __syncthreads();
        if (th.F < 0) continue;      // outputs of that set are copies of f: no neighbour terms

        const Pair* pr = a.pairs + (size_t)tset * a.cap_pairs;
        const int K = th.F + th.z;
        for (int k = 0; k < K; ++k) {
            float om_hi = 0.f, om_lo = 0.f, Wk = th.w0;
            if (k < th.F) {
                const Pair p = pr[k];
                om_hi = p.om_hi;
                om_lo = p.om_lo;
                Wk = p.W;
            }
            fir32::PhaseSteps<PS, 0, PS::ITERS>::run(ps, fz, cs, a.H, om_hi, om_lo);
            __syncthreads();
            // forward planes (A, B) = G(f'c, f's), (C, D) = G(c, s) at my outputs
            // (centre terms, own set only)
            float2 fAB[8], fCD[8];
            if (own) {
                fir32::row_pass_2x2<G, NCH, NT, true>(tp2, cs, fz, fz, hz1, hz2, tid);
                __syncthreads();
                fir32::col_pass_2x2<NCH>(tp2, hz1, hz2, o, rb, fAB, fCD);
                __syncthreads();
            }
            // adjoint planes (G(ac), G(as)), (G(bc), G(bs)) at my outputs
            fir32::row_pass_2x2<G, NCH, NT, false>(tp2, cs, az, bz, hz1, hz2, tid);
            __syncthreads();
            float2 gA[8], gB[8];
            fir32::col_pass_2x2<NCH>(tp2, hz1, hz2, o, rb, gA, gB);
            const float w = om_hi;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = rb * 8 + i + Rp, col = o + Rp;
                const float2 cc = cs[r * G::CSp + col];
                const float c = cc.x, s = cc.y, fc = fz[r * G::FP + col];
                const float Gac = gA[i].x, Gas = gA[i].y, Gbc = gB[i].x, Gbs = gB[i].y;
                float v = fmaf(c, Gac, s * Gas);
                v = fmaf(-w * fc, fmaf(s, Gac, -c * Gas), v);
                v = fmaf(-w, fmaf(s, Gbc, -c * Gbs), v);
                if (own) {
                    const float av = az[r * G::FP + col], bv = bz[r * G::FP + col];
                    v = fmaf(w * av, fmaf(c, fAB[i].y, -s * fAB[i].x), v);
                    v = fmaf(w * bv, fmaf(c, fCD[i].y, -s * fCD[i].x), v);
                }
                grad[i] = fmaf(Wk, v, grad[i]);
            }
            __syncthreads();
        }
    }

    if (gx < a.W) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gy = by + rb * 8 + i;
            if (gy >= a.H) continue;
            const int r = rb * 8 + i + Rp;
            const size_t k = (size_t)gy * a.pitch + gx;
            float g = grad[i];
            // out = f where the guard fired or the set passed the image through
            if (hd.F < 0 || !(a.den[(size_t)gy * a.spitch + gx] > kGuard * rmass[r] * cmass[o + Rp]))
                g += __ldg(a.u + k);
            a.grad[k] = g;
        }
    }
}

template <int NCH>
cudaError_t launch_packed(const BwdArgs& a, cudaStream_t s)
{
    constexpr int TH = 64;
    constexpr size_t smem = BwdGeo<TH, NCH>::bytes;
    const int Rp = 4 * (NCH - 1);
    fir32::Taps2 tp2;
    for (int i = 0; i < (int)(sizeof(tp2.g) / sizeof(float2)); ++i) {
        const int k = i - 8 - Rp;
        const float g = (k >= -a.R && k <= a.R) ? a.h_taps[k + a.R] : 0.f;
        tp2.g[i] = make_float2(g, g);
    }
    cudaError_t e = cudaFuncSetAttribute(k_bwd32x<TH, NCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + 31) / 32, (a.H + TH - 1) / TH);
    k_bwd32x<TH, NCH><<<grid, TH * 4, smem, s>>>(a, tp2);
    return cudaGetLastError();
}

size_t bwd_smem(int R, int th, int tw)
{
    const Geo G(R, th, tw);
    return (G.floats(tw, 5) + G.RH + G.RW) * sizeof(float);
}

template <int TH, int TW>
cudaError_t launch_tile(const BwdArgs& a, cudaStream_t s)
{
    const size_t smem = bwd_smem(a.R, TH, TW);
    cudaError_t e = cudaFuncSetAttribute(k_bwd32<TH, TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    k_bwd32<TH, TW><<<grid, TH * TW / 8, smem, s>>>(a);
    return cudaGetLastError();
}

constexpr size_t kSmemLimit = 227 * 1024;

}  // namespace

void bwd32_tile(int R, int* th, int* tw)
{
    static const int shapes[][2] = {{64, 32}, {32, 32}, {16, 16}};
    for (auto& sh : shapes)
        if (bwd_smem(R, sh[0], sh[1]) <= kSmemLimit) {
            *th = sh[0];
            *tw = sh[1];
            return;
        }
    *th = *tw = 0;
}

cudaError_t launch_bwd32(const BwdArgs& a, cudaStream_t s)
{
    if (a.h_taps && a.R >= 1) {
        switch ((a.R + 3) / 4 + 1) {      // NCH = Rp / 4 + 1, Rp <= 20
            case 2: return launch_packed<2>(a, s);
            case 3: return launch_packed<3>(a, s);
            case 4: return launch_packed<4>(a, s);
            case 5: return launch_packed<5>(a, s);
            case 6: return launch_packed<6>(a, s);
            default: break;
        }
    }
    int th, tw;
    bwd32_tile(a.R, &th, &tw);
    if (th == 64 && tw == 32) return launch_tile<64, 32>(a, s);
    if (th == 32 && tw == 32) return launch_tile<32, 32>(a, s);
    if (th == 16 && tw == 16) return launch_tile<16, 16>(a, s);
    return cudaErrorNotSupported;
}

}  // namespace bf
