// FP32 building blocks of the SIMT kernels (forward K3 and adjoint K5):
// accurate phases and the register-blocked separable FIR over a tile + halo
// staged in shared memory.
#pragma once

#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace fir32 {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float k2PiHi = (float)kTwoPi;
constexpr float k2PiLo = (float)(kTwoPi - (double)(float)kTwoPi);
constexpr float kInv2Pi = (float)(1.0 / kTwoPi);

// cos and sin of (om_hi + om_lo) * v: the product is formed as head + exact
// tail (FMA TwoProduct, Ogita-Rump-Oishi 2005), reduced by 2 pi with a
// two-part constant (Cody-Waite 1980) and evaluated on the SFU.
__device__ __forceinline__ void phase_cs(float v, float om_hi, float om_lo, float& c, float& s)
{
    const float p = __fmul_rn(om_hi, v);
    float e = fmaf(om_hi, v, -p);           // exact rounding error of p
    e = fmaf(om_lo, v, e);                  // + tail of omega
    const float q = rintf(__fmul_rn(p, kInv2Pi));
    float r = fmaf(-q, k2PiHi, p);
    r = fmaf(-q, k2PiLo, r);
    r = __fadd_rn(r, e);
    __sincosf(r, &s, &c);
}

// Element j (0..7, a compile-time constant after unrolling) of the pair (a, b).
__device__ __forceinline__ float pick8(const float4& a, const float4& b, int j)
{
    switch (j) {
    case 0: return a.x;
    case 1: return a.y;
    case 2: return a.z;
    case 3: return a.w;
    case 4: return b.x;
    case 5: return b.y;
    case 6: return b.z;
    default: return b.w;
    }
}

// Shared-memory geometry for a tile of TH x TW outputs and radius R.
struct Geo {
    int R, nch, RH, RW, RWp, RHp, ngz;
    __host__ __device__ Geo(int R_, int TH, int TW)
    {
        R = R_;
        nch = (2 * R + 15) / 8;                 // 8-wide steps covering 2R+8 inputs
        RH = TH + 2 * R;
        RW = TW + 2 * R;
        RWp = TW - 8 + 8 * nch + 4;             // +4 words: rows 16 B aligned, banks staggered
        RHp = TH - 8 + 8 * nch;
        ngz = 8 * nch + 16;
    }
    // floats of shared memory with `region` halo-sized arrays and 4 row-filtered planes
    __host__ __device__ size_t floats(int TW, int region) const
    {
        return (size_t)region * RH * RWp + 4 * (size_t)RHp * TW + (size_t)ngz;
    }
};

// Row pass: for every halo row r and 8-column block cb of the tile, the 4
// planes (m1 c, m1 s, m2 c, m2 s) -- or (m1 c, m1 s, c, s) when kOnes --
// filtered with the 2R+1 taps, written to hsm (4 planes of RHp x TW).
// Register-blocked: 8 outputs per thread, 8 inputs per step; the taps array
// gz is zero outside [0, 2R] so that no branch guards the window.
template <int TW, bool kOnes>
__device__ __forceinline__ void row_pass(const Geo& G, const float* m1s, const float* m2s,
                                         const float* csm, const float* ssm, const float* gz,
                                         float* hsm, int tid, int nthreads)
{
    const size_t hplane = (size_t)G.RHp * TW;
    for (int it = tid; it < G.RH * (TW / 8); it += nthreads) {
        const int r = it / (TW / 8), cb = it - r * (TW / 8);
        const float* ar = m1s + r * G.RWp + cb * 8;
        const float* br = m2s + r * G.RWp + cb * 8;
        const float* cr = csm + r * G.RWp + cb * 8;
        const float* sr = ssm + r * G.RWp + cb * 8;
        float acc[4][8];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[q][i] = 0.f;
        for (int ch = 0; ch < G.nch; ++ch) {
            const int a0 = ch * 8;
            float g[15];
#pragma unroll
            for (int d = 0; d < 15; ++d) g[d] = gz[a0 + d + 1];   // tap a0 + d - 7
            const float4 c0 = *(const float4*)(cr + a0), c1 = *(const float4*)(cr + a0 + 4);
            const float4 s0 = *(const float4*)(sr + a0), s1 = *(const float4*)(sr + a0 + 4);
            const float4 f0 = *(const float4*)(ar + a0), f1 = *(const float4*)(ar + a0 + 4);
            float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
            if (!kOnes) {
                b0 = *(const float4*)(br + a0);
                b1 = *(const float4*)(br + a0 + 4);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float cj = pick8(c0, c1, j), sj = pick8(s0, s1, j);
                const float fj = pick8(f0, f1, j);
                const float A = fj * cj, B = fj * sj;
                float C = cj, D = sj;
                if (!kOnes) {
                    const float bj = pick8(b0, b1, j);
                    C = bj * cj;
                    D = bj * sj;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float w = g[j - i + 7];
                    acc[0][i] = fmaf(w, A, acc[0][i]);
                    acc[1][i] = fmaf(w, B, acc[1][i]);
                    acc[2][i] = fmaf(w, C, acc[2][i]);
                    acc[3][i] = fmaf(w, D, acc[3][i]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float* hp = hsm + q * hplane + (size_t)r * TW + cb * 8;
            *(float4*)hp = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
            *(float4*)(hp + 4) = make_float4(acc[q][4], acc[q][5], acc[q][6], acc[q][7]);
        }
    }
}

// Column pass of one thread's item: column o, output rows rb*8 .. rb*8+7.
template <int TW>
__device__ __forceinline__ void col_pass(const Geo& G, const float* hsm, const float* gz, int o,
                                         int rb, float (&acc)[4][8])
{
    const size_t hplane = (size_t)G.RHp * TW;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[q][i] = 0.f;
    const float* h0 = hsm + (size_t)(rb * 8) * TW + o;
    for (int ch = 0; ch < G.nch; ++ch) {
        const int a0 = ch * 8;
        float g[15];
#pragma unroll
        for (int d = 0; d < 15; ++d) g[d] = gz[a0 + d + 1];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float* hj = h0 + (size_t)(a0 + j) * TW;
            const float hA = hj[0], hB = hj[hplane], hC = hj[2 * hplane], hD = hj[3 * hplane];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float w = g[j - i + 7];
                acc[0][i] = fmaf(w, hA, acc[0][i]);
                acc[1][i] = fmaf(w, hB, acc[1][i]);
                acc[2][i] = fmaf(w, hC, acc[2][i]);
                acc[3][i] = fmaf(w, hD, acc[3][i]);
            }
        }
    }
}

}  // namespace fir32
}  // namespace bf

namespace bf {
namespace fir32 {

// ---- tall-tile variant: two row-filtered planes at a time, exact taps ------
//
// The radius is padded to Rp = 4 ceil(R/4) (taps beyond R are zero and add
// exact zeros), so that 2 Rp is a multiple of 8: the first 8-input step of
// an 8-output block then only meets taps j - i >= 0 (lower triangle) and the
// last one only taps j - i <= 0 (upper triangle), and the FIR executes
// exactly 2 Rp + 1 multiply-adds per output.  The row-filtered planes are
// stored with the 16-byte quads of each row permuted by (row & 7), which
// spreads the vector stores of a warp over all 32 banks.

struct Geo2 {
    int R, Rp, nch, RH, RW, RWp, RHp, ngz;
    __host__ __device__ Geo2(int R_, int TH, int TW)
    {
        R = R_;
        Rp = (R + 3) / 4 * 4;
        nch = Rp / 4 + 1;                       // (2 Rp + 8) / 8 input steps
        RH = TH + 2 * Rp;
        RW = TW + 2 * Rp;
        RWp = TW - 8 + 8 * nch + 4;             // = RW + 4: rows 16 B aligned, banks staggered
        RHp = TH - 8 + 8 * nch;                 // = RH
        ngz = 8 * nch + 16;
    }
    // the sin array and the second row-filtered plane start 4 words (16 B)
    // past a bank-aligned offset, so that the two arrays a quarter-warp
    // reads or writes together fall on different banks
    __host__ __device__ size_t region() const { return (size_t)RH * RWp; }
    __host__ __device__ size_t hplane(int TW) const { return (size_t)RHp * TW + 4; }
    __host__ __device__ size_t floats(int TW) const
    {
        return 3 * region() + 4 + 2 * hplane(TW) + (size_t)ngz;
    }
};

// word offset of element (row r, column x) of a swizzled row-filtered plane
template <int TW>
__device__ __forceinline__ int hsw(int r, int x)
{
    return r * TW + ((((x >> 2) ^ (r & 7)) & (TW / 4 - 1)) << 2) + (x & 3);
}

// One 8x8 step of an 8-output FIR block: acc[i] += g[j - i + 7] * v[j] for
// the (j, i) allowed by kPart (0 full, 1 lower triangle j >= i, 2 upper j <= i).
template <int kPart>
__device__ __forceinline__ void fir_step(float (&acc)[8], const float (&g)[15], const float (&v)[8])
{
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (kPart == 1 && j < i) continue;
            if (kPart == 2 && j > i) continue;
            acc[i] = fmaf(g[j - i + 7], v[j], acc[i]);
        }
}

// Row pass for one plane per item: plane value m * cs (m = m1s, or 1 when
// m1s is null), items (halo row r, 8-column block cb, plane p of the pair
// (p = 0 uses cos, p = 1 sin)); output to hsm plane p (swizzled rows).
template <int TW>
__device__ __forceinline__ void row_pass2(const Geo2& G, const float* m1s, const float* csm,
                                          const float* ssm, const float* gz, float* hsm, int tid,
                                          int nthreads)
{
    const size_t hplane = G.hplane(TW);
    for (int it = tid; it < G.RH * (TW / 8) * 2; it += nthreads) {
        const int p = it & 1, rc = it >> 1;
        const int r = rc / (TW / 8), cb = rc - r * (TW / 8);
        const float* src = (p ? ssm : csm) + r * G.RWp + cb * 8;
        const float* mr = m1s ? m1s + r * G.RWp + cb * 8 : nullptr;
        float acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = 0.f;
        for (int ch = 0; ch < G.nch; ++ch) {
            const int a0 = ch * 8;
            float g[15];
#pragma unroll
            for (int d = 0; d < 15; ++d) g[d] = gz[a0 + d + 1];   // tap a0 + d - 7
            const float4 v0 = *(const float4*)(src + a0), v1 = *(const float4*)(src + a0 + 4);
            float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            if (mr) {
                const float4 f0 = *(const float4*)(mr + a0), f1 = *(const float4*)(mr + a0 + 4);
                v[0] *= f0.x; v[1] *= f0.y; v[2] *= f0.z; v[3] *= f0.w;
                v[4] *= f1.x; v[5] *= f1.y; v[6] *= f1.z; v[7] *= f1.w;
            }
            if (ch == 0) fir_step<1>(acc, g, v);
            else if (ch == G.nch - 1) fir_step<2>(acc, g, v);
            else fir_step<0>(acc, g, v);
        }
        float* hp = hsm + p * hplane;
        *(float4*)(hp + hsw<TW>(r, cb * 8)) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        *(float4*)(hp + hsw<TW>(r, cb * 8 + 4)) = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
}

// Column pass of two planes for one item: column o, output rows rb*8 .. rb*8+7.
template <int TW>
__device__ __forceinline__ void col_pass2(const Geo2& G, const float* hsm, const float* gz, int o,
                                          int rb, float (&acc)[2][8])
{
    const size_t hplane = G.hplane(TW);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[q][i] = 0.f;
    for (int ch = 0; ch < G.nch; ++ch) {
        const int a0 = ch * 8;
        float g[15];
#pragma unroll
        for (int d = 0; d < 15; ++d) g[d] = gz[a0 + d + 1];
        float v0[8], v1[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = rb * 8 + a0 + j;
            const int w = hsw<TW>(r, o);
            v0[j] = hsm[w];
            v1[j] = hsm[hplane + w];
        }
        if (ch == 0) {
            fir_step<1>(acc[0], g, v0);
            fir_step<1>(acc[1], g, v1);
        } else if (ch == G.nch - 1) {
            fir_step<2>(acc[0], g, v0);
            fir_step<2>(acc[1], g, v1);
        } else {
            fir_step<0>(acc[0], g, v0);
            fir_step<0>(acc[1], g, v1);
        }
    }
}

}  // namespace fir32
}  // namespace bf

namespace bf {
namespace fir32 {

// ---- compile-time tap count: taps as kernel parameters ---------------------
//
// With NCH (the number of 8-input steps, Rp / 4 + 1) a template parameter the
// FIR loops unroll completely and every tap index is a constant, so the taps
// are read from the kernel's parameter bank as FFMA operands instead of being
// loaded from shared memory.  R >= 1 makes NCH >= 2, so the first and last
// steps are distinct.

constexpr int kTapsMaxRp = 24;    // the tall tile's largest padded radius
struct Taps {
    float g[8 * (kTapsMaxRp / 4 + 1) + 16];   // g[t + 8] = g(t - Rp), 0 outside |t - Rp| <= R
};

template <int TW, int NCH>
__device__ __forceinline__ void row_pass2c(const Geo2& G, const Taps& tp, const float* m1s,
                                           const float* csm, const float* ssm, float* hsm,
                                           int tid, int nthreads)
{
    const size_t hplane = G.hplane(TW);
    for (int it = tid; it < G.RH * (TW / 8) * 2; it += nthreads) {
        const int p = it & 1, rc = it >> 1;
        const int r = rc / (TW / 8), cb = rc - r * (TW / 8);
        const float* src = (p ? ssm : csm) + r * G.RWp + cb * 8;
        const float* mr = m1s ? m1s + r * G.RWp + cb * 8 : nullptr;
        float acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            const int a0 = ch * 8;
            float g[15];
#pragma unroll
            for (int d = 0; d < 15; ++d) g[d] = tp.g[a0 + d + 1];
            const float4 v0 = *(const float4*)(src + a0), v1 = *(const float4*)(src + a0 + 4);
            float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            if (mr) {
                const float4 f0 = *(const float4*)(mr + a0), f1 = *(const float4*)(mr + a0 + 4);
                v[0] *= f0.x; v[1] *= f0.y; v[2] *= f0.z; v[3] *= f0.w;
                v[4] *= f1.x; v[5] *= f1.y; v[6] *= f1.z; v[7] *= f1.w;
            }
            if (ch == 0) {
                fir_step<1>(acc, g, v);
            } else if (ch == NCH - 1) {
                fir_step<2>(acc, g, v);
            } else {
                fir_step<0>(acc, g, v);
            }
        }
        float* hp = hsm + p * hplane;
        *(float4*)(hp + hsw<TW>(r, cb * 8)) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        *(float4*)(hp + hsw<TW>(r, cb * 8 + 4)) = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
}

template <int TW, int NCH>
__device__ __forceinline__ void col_pass2c(const Geo2& G, const Taps& tp, const float* hsm, int o,
                                           int rb, float (&acc)[2][8])
{
    const size_t hplane = G.hplane(TW);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[q][i] = 0.f;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        const int a0 = ch * 8;
        float g[15];
#pragma unroll
        for (int d = 0; d < 15; ++d) g[d] = tp.g[a0 + d + 1];
        float v0[8], v1[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = rb * 8 + a0 + j;
            const int w = hsw<TW>(r, o);
            v0[j] = hsm[w];
            v1[j] = hsm[hplane + w];
        }
        if (ch == 0) {
            fir_step<1>(acc[0], g, v0);
            fir_step<1>(acc[1], g, v1);
        } else if (ch == NCH - 1) {
            fir_step<2>(acc[0], g, v0);
            fir_step<2>(acc[1], g, v1);
        } else {
            fir_step<0>(acc[0], g, v0);
            fir_step<0>(acc[1], g, v1);
        }
    }
}

}  // namespace fir32
}  // namespace bf
