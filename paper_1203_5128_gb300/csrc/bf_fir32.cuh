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

// ---- tall tile, packed pairs: the cos and sin planes of a pass ride in one
// 64-bit register pair and advance together in packed FP32 multiply-adds
// (fma.rn.f32x2, sm_100 and later), which halves the issue slots of the FIR.
//
// The radius is padded to Rp = 4 ceil(R/4) (taps beyond R are zero and add
// exact zeros), so that 2 Rp is a multiple of 8: the first 8-input step of an
// 8-output block then only meets taps j - i >= 0 (lower triangle) and the
// last one only taps j - i <= 0 (upper triangle), and the FIR executes exactly
// 2 Rp + 1 multiply-adds per output.  With NCH (the number of 8-input steps,
// Rp / 4 + 1) a template parameter the FIR loops unroll completely, every tap
// index is a constant and the taps are read from the kernel's parameter bank.
//
// Shared memory (NCH fixes every size):
//   cs   RH x CSp float2   (cos, sin) of the halo pixels; CSp = RW + 2 makes a
//                           row an odd number of 16-byte chunks, so the eight
//                           rows a quarter-warp reads fall on distinct banks;
//   fz   RH x FP  float    centred f; FP = RW + 4, an odd number of chunks;
//   hz   RH x TW  float2   row-filtered pair, 16-byte chunks of row r
//                           permuted by (r & 7).

constexpr int kTapsMaxRp = 24;    // the tall tile's largest padded radius
struct Taps {
    float g[8 * (kTapsMaxRp / 4 + 1) + 16];   // g[t + 8] = g(t - Rp), 0 outside |t - Rp| <= R
};
struct Taps2 {
    float2 g[8 * (kTapsMaxRp / 4 + 1) + 16];  // (g, g) with g as in Taps
};

template <int TH, int TW, int NCH>
struct TallGeo {
    static constexpr int Rp = 4 * (NCH - 1);
    static constexpr int RH = TH + 2 * Rp;
    static constexpr int RW = TW + 2 * Rp;
    static constexpr int CSp = RW + 2;
    static constexpr int FP = RW + 4;
    static constexpr size_t cs_bytes = (size_t)RH * CSp * 8;
    static constexpr size_t fz_bytes = (size_t)RH * FP * 4;
    static constexpr size_t hz_bytes = (size_t)RH * TW * 8;
    static constexpr size_t bytes = cs_bytes + fz_bytes + hz_bytes;
    static_assert(TW == 32, "the swizzle assumes 16 chunks per row-filtered row");
    static_assert(RH % 8 == 0 && (CSp / 2) % 2 == 1 && (FP / 4) % 2 == 1, "bank layout");
};

// float2 index of element (row r, column x) of the swizzled row-filtered pair
__device__ __forceinline__ int hz_at(int r, int x)
{
    return r * 32 + ((((x >> 1) ^ (r & 7)) << 1) | (x & 1));
}

// One input step on pairs: acc[i] += g(d - Rp) v[j] with d = s0 + j - i, for
// the (j, i) whose d lies in [0, 2 Rp]; s0 is a compile-time constant after
// unrolling, so the window test costs nothing and tp.g[d + 8] is a constant-
// bank operand.
template <int NO, int NI, int Rp>
__device__ __forceinline__ void fir_x2(float2 (&acc)[NO], const Taps2& tp, int s0,
                                       const float2 (&v)[NI])
{
#pragma unroll
    for (int j = 0; j < NI; ++j)
#pragma unroll
        for (int i = 0; i < NO; ++i) {
            const int d = s0 + j - i;
            if (d < 0 || d > 2 * Rp) continue;
            acc[i] = __ffma2_rn(tp.g[d + 8], v[j], acc[i]);
        }
}

// Row FIR of NO consecutive outputs (NO = 4 or 8) of a pair plane: inputs
// src[0 .. NO + 2 Rp), in steps of NO.
template <int NO, int NCH>
__device__ __forceinline__ void row_item_x2(const Taps2& tp, const float2* src, float2 (&acc)[NO])
{
    constexpr int Rp = 4 * (NCH - 1), NS = (NO + 2 * Rp) / NO;
#pragma unroll
    for (int i = 0; i < NO; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        float2 v[NO];
#pragma unroll
        for (int q = 0; q < NO / 2; ++q) {
            const float4 w = *(const float4*)(src + st * NO + 2 * q);
            v[2 * q] = make_float2(w.x, w.y);
            v[2 * q + 1] = make_float2(w.z, w.w);
        }
        fir_x2<NO, NO, Rp>(acc, tp, st * NO, v);
    }
}

// Box filter (taps 1 inside [-R, R], 0 outside) on NO consecutive outputs
// of a pair plane: the first output is the FIR sum of its window (the same
// taps in the same order as row_item_x2), each next one the previous plus
// the value entering the window minus the value leaving it.  The sliding sum
// restarts every NO outputs, so an output carries at most 2 (NO - 1)
// roundings more than the direct sum of its 2R + 1 values.
template <int NO, int NCH>
__device__ __forceinline__ void row_item_box_x2(const Taps2& tp, const float2* src, int R,
                                                float2 (&acc)[NO])
{
    constexpr int Rp = 4 * (NCH - 1);
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q <= Rp; ++q) {       // inputs 2q, 2q + 1 (the last one, 2 Rp + 1, unused)
        const float4 w = *(const float4*)(src + 2 * q);
        s = __ffma2_rn(tp.g[2 * q + 8], make_float2(w.x, w.y), s);
        if (2 * q + 1 <= 2 * Rp) s = __ffma2_rn(tp.g[2 * q + 9], make_float2(w.z, w.w), s);
    }
    acc[0] = s;
#pragma unroll
    for (int i = 1; i < NO; ++i) {
        s = __fadd2_rn(s, src[i + Rp + R]);
        s = __ffma2_rn(make_float2(-1.f, -1.f), src[i - 1 + Rp - R], s);
        acc[i] = s;
    }
}

// Box row run of NO outputs (even) stored into hz as they are formed: the
// window's FIR sum for the first output, then sliding sums as in
// row_item_box_x2 (no accumulator array, so the run can be a whole row).
template <int NO, int NCH>
__device__ __forceinline__ void row_run_box_x2(const Taps2& tp, const float2* src, int R,
                                               float2* hz, int r, int x0)
{
    constexpr int Rp = 4 * (NCH - 1);
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q <= Rp; ++q) {
        const float4 w = *(const float4*)(src + 2 * q);
        s = __ffma2_rn(tp.g[2 * q + 8], make_float2(w.x, w.y), s);
        if (2 * q + 1 <= 2 * Rp) s = __ffma2_rn(tp.g[2 * q + 9], make_float2(w.z, w.w), s);
    }
    float2 prev = s;
#pragma unroll
    for (int i = 1; i < NO; ++i) {
        s = __fadd2_rn(s, src[i + Rp + R]);
        s = __ffma2_rn(make_float2(-1.f, -1.f), src[i - 1 + Rp - R], s);
        if (i & 1) *(float4*)(hz + hz_at(r, x0 + i - 1)) = make_float4(prev.x, prev.y, s.x, s.y);
        prev = s;
    }
}

// Row pass of a pair plane into the swizzled hz (kBox: the sliding box sums
// of row_run_box_x2 for radius R, one run per row).  The first NT-multiple of the
// RH x 4 items (halo row r, 8-column block) runs as 8-output items, the
// eight rows of a quarter-warp consecutive; the rest runs, when it fits one
// round that way, as twice as many 4-output items (the last round then takes
// half as long), else as 8-output items too.
template <int TH, int TW, int NCH, int NT, bool kBox = false>
__device__ __forceinline__ void row_pass_x2(const Taps2& tp, const float2* cs, float2* hz, int tid,
                                            int R = 0)
{
    using G = TallGeo<TH, TW, NCH>;
    constexpr int kItems = G::RH * (TW / 8);
    constexpr int kFull = kItems / NT * NT;
    constexpr bool kSplit = 2 * (kItems - kFull) <= NT;
    constexpr int kMain = kSplit ? kFull : kItems;
    constexpr int kHalf = kSplit ? 2 * (kItems - kFull) : 0;
    static_assert(kItems % 32 == 0 && kFull % 32 == 0, "row pass items");
    if constexpr (kBox) {
        // box: one run per row, so that each window's direct sum serves the
        // row's 32 sliding outputs (consecutive threads on consecutive rows)
        for (int r = tid; r < G::RH; r += NT) row_run_box_x2<TW, NCH>(tp, cs + r * G::CSp, R, hz, r, 0);
        return;
    }
    for (int it = tid; it < kMain; it += NT) {
        const int cb = (it >> 3) & 3, r = (it & 7) + ((it >> 5) << 3);
        float2 acc[8];
        if constexpr (kBox) row_item_box_x2<8, NCH>(tp, cs + r * G::CSp + cb * 8, R, acc);
        else row_item_x2<8, NCH>(tp, cs + r * G::CSp + cb * 8, acc);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *(float4*)(hz + hz_at(r, cb * 8 + 2 * q)) =
                make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y);
    }
    if (kHalf > 0 && tid < kHalf) {
        const int r = kFull / 4 + (tid & 7) + ((tid >> 6) << 3), x0 = ((tid >> 3) & 7) * 4;
        float2 acc[4];
        if constexpr (kBox) row_item_box_x2<4, NCH>(tp, cs + r * G::CSp + x0, R, acc);
        else row_item_x2<4, NCH>(tp, cs + r * G::CSp + x0, acc);
#pragma unroll
        for (int q = 0; q < 2; ++q)
            *(float4*)(hz + hz_at(r, x0 + 2 * q)) =
                make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y);
    }
}

// Row FIR of NO outputs for two pairs: (m1 c, m1 s) and (m2 c, m2 s), m2 = 1
// when kOnes.
template <int NO, int NCH, bool kOnes>
__device__ __forceinline__ void row_item_2x2(const Taps2& tp, const float2* src, const float* m1,
                                             const float* m2, float2 (&acc1)[NO],
                                             float2 (&acc2)[NO])
{
    constexpr int Rp = 4 * (NCH - 1), NS = (NO + 2 * Rp) / NO;
#pragma unroll
    for (int i = 0; i < NO; ++i) acc1[i] = acc2[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        float2 v[NO], va[NO], vb[NO];
#pragma unroll
        for (int q = 0; q < NO / 2; ++q) {
            const float4 w = *(const float4*)(src + st * NO + 2 * q);
            v[2 * q] = make_float2(w.x, w.y);
            v[2 * q + 1] = make_float2(w.z, w.w);
        }
#pragma unroll
        for (int q = 0; q < NO / 4; ++q) {
            const float4 m = *(const float4*)(m1 + st * NO + 4 * q);
            va[4 * q] = __fmul2_rn(make_float2(m.x, m.x), v[4 * q]);
            va[4 * q + 1] = __fmul2_rn(make_float2(m.y, m.y), v[4 * q + 1]);
            va[4 * q + 2] = __fmul2_rn(make_float2(m.z, m.z), v[4 * q + 2]);
            va[4 * q + 3] = __fmul2_rn(make_float2(m.w, m.w), v[4 * q + 3]);
            if (kOnes) {
                vb[4 * q] = v[4 * q];
                vb[4 * q + 1] = v[4 * q + 1];
                vb[4 * q + 2] = v[4 * q + 2];
                vb[4 * q + 3] = v[4 * q + 3];
            } else {
                const float4 n = *(const float4*)(m2 + st * NO + 4 * q);
                vb[4 * q] = __fmul2_rn(make_float2(n.x, n.x), v[4 * q]);
                vb[4 * q + 1] = __fmul2_rn(make_float2(n.y, n.y), v[4 * q + 1]);
                vb[4 * q + 2] = __fmul2_rn(make_float2(n.z, n.z), v[4 * q + 2]);
                vb[4 * q + 3] = __fmul2_rn(make_float2(n.w, n.w), v[4 * q + 3]);
            }
        }
        fir_x2<NO, NO, Rp>(acc1, tp, st * NO, va);
        fir_x2<NO, NO, Rp>(acc2, tp, st * NO, vb);
    }
}

template <int NO>
__device__ __forceinline__ void store_row_x2(float2* hz, int r, int x0, const float2 (&acc)[NO])
{
#pragma unroll
    for (int q = 0; q < NO / 2; ++q)
        *(float4*)(hz + hz_at(r, x0 + 2 * q)) =
            make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y);
}

// Row pass of two pairs into the swizzled planes hz1, hz2 (TW = 32, rows of
// the halo RH, pitches CSp / FP of the geometry G).  Items (halo row, 8-column
// block), the eight rows of a quarter-warp consecutive: full rounds of
// 8-output items, then the rest as twice as many 4-output items when they
// fit one round, else as 8-output items.
template <class G, int NCH, int NT, bool kOnes>
__device__ __forceinline__ void row_pass_2x2(const Taps2& tp, const float2* cs, const float* m1,
                                             const float* m2, float2* hz1, float2* hz2, int tid)
{
    constexpr int TW = 32;
    constexpr int kItems = G::RH * (TW / 8);
    constexpr int kFull = kItems / NT * NT;
    constexpr bool kSplit = 2 * (kItems - kFull) <= NT;
    constexpr int kMain = kSplit ? kFull : kItems;
    constexpr int kHalf = kSplit ? 2 * (kItems - kFull) : 0;
    static_assert(kItems % 32 == 0 && kFull % 32 == 0, "row pass items");
    for (int it = tid; it < kMain; it += NT) {
        const int cb = (it >> 3) & 3, r = (it & 7) + ((it >> 5) << 3);
        float2 acc1[8], acc2[8];
        row_item_2x2<8, NCH, kOnes>(tp, cs + r * G::CSp + cb * 8, m1 + r * G::FP + cb * 8,
                                    m2 + r * G::FP + cb * 8, acc1, acc2);
        store_row_x2<8>(hz1, r, cb * 8, acc1);
        store_row_x2<8>(hz2, r, cb * 8, acc2);
    }
    if (kHalf > 0 && tid < kHalf) {
        const int r = kFull / 4 + (tid & 7) + ((tid >> 6) << 3), x0 = ((tid >> 3) & 7) * 4;
        float2 acc1[4], acc2[4];
        row_item_2x2<4, NCH, kOnes>(tp, cs + r * G::CSp + x0, m1 + r * G::FP + x0,
                                    m2 + r * G::FP + x0, acc1, acc2);
        store_row_x2<4>(hz1, r, x0, acc1);
        store_row_x2<4>(hz2, r, x0, acc2);
    }
}

// Column pass of two pairs for one item: column o, output rows rb*8 .. rb*8+7.
template <int NCH>
__device__ __forceinline__ void col_pass_2x2(const Taps2& tp, const float2* hz1, const float2* hz2,
                                             int o, int rb, float2 (&acc1)[8], float2 (&acc2)[8])
{
    constexpr int Rp = 4 * (NCH - 1), NS = NCH;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc1[i] = acc2[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int ch = 0; ch < NS; ++ch) {
        float2 v1[8], v2[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int w = hz_at(rb * 8 + ch * 8 + j, o);
            v1[j] = hz1[w];
            v2[j] = hz2[w];
        }
        fir_x2<8, 8, Rp>(acc1, tp, ch * 8, v1);
        fir_x2<8, 8, Rp>(acc2, tp, ch * 8, v2);
    }
}

// Phase sweep of a tile (geometry G: RH x RW halo, cs / fz pitches CSp / FP):
// the first S * RW threads own one halo column
// each (col = tid % RW) and rows r0 + S m, r0 = tid / RW, m = 0 .. ITERS-1, so
// that every shared-memory address is a per-thread base plus a constant.
template <class G, int NT>
struct PhaseSweep {
    static constexpr int S = NT / G::RW;
    static constexpr int ITERS = (G::RH + S - 1) / S;
    bool on, x_in;
    int r0, fbase, cbase, gyb;
    __device__ __forceinline__ PhaseSweep(int tid, int gy0, int gx0, int W)
    {
        on = tid < S * G::RW;
        r0 = tid / G::RW;
        const int col = tid - r0 * G::RW;
        x_in = (unsigned)(gx0 + col) < (unsigned)W;
        fbase = r0 * G::FP + col;
        cbase = r0 * G::CSp + col;
        gyb = gy0 + r0;
    }
    // (cos, sin) of row r0 + S m for the frequency (om_hi + om_lo); zero outside the image
    template <int m>
    __device__ __forceinline__ void step(const float* fz, float2* cs, int H, float om_hi,
                                         float om_lo) const
    {
        if (m >= ITERS) return;
        if (!on || (m == ITERS - 1 && r0 + S * m >= G::RH)) return;
        float c, sn;
        phase_cs(fz[fbase + S * m * G::FP], om_hi, om_lo, c, sn);
        const bool in = x_in && (unsigned)(gyb + S * m) < (unsigned)H;
        cs[cbase + S * m * G::CSp] = in ? make_float2(c, sn) : make_float2(0.f, 0.f);
    }
};

template <class PS, int m0, int n>
struct PhaseSteps {
    __device__ __forceinline__ static void run(const PS& ps, const float* fz, float2* cs, int H,
                                               float om_hi, float om_lo)
    {
        ps.template step<m0>(fz, cs, H, om_hi, om_lo);
        PhaseSteps<PS, m0 + 1, n - 1>::run(ps, fz, cs, H, om_hi, om_lo);
    }
};
template <class PS, int m0>
struct PhaseSteps<PS, m0, 0> {
    __device__ __forceinline__ static void run(const PS&, const float*, float2*, int, float, float) {}
};

}  // namespace fir32
}  // namespace bf
