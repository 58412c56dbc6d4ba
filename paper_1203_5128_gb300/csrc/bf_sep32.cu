// K3-sep: the FP32 FIR forward (Sec. 1.2, eqs. (f1)-(f2)) in two passes
// through HBM, for radii whose halo does not fit a fused tile (R > 24) in
// plans with one parameter set.
//
// The fused kernels keep a tile and its 2R halo in shared memory; beyond
// R = 24 only 32 x 32 or 16 x 16 tiles fit, and their halo work grows to
// 7-50 times the outputs.  Here the two separable passes meet in HBM:
//
//   k_sep_rows  a CTA takes 8 image rows x 128 output columns (+ R halo
//               columns): f once, then per term its phases and the pairs
//               (f'c, f's), (c, s) filtered along the row as packed pairs
//               (fma.rn.f32x2; 8 outputs x 8 inputs per register-blocked
//               step, taps as constant-bank operands), written to a buffer of
//               nk terms, [term][pair][H][Wp] float2;
//   k_sep_cols  a CTA takes 128 x 32 outputs: per term and pair, the
//               (128 + 2R) x 32 column strip arrives by cp.async in a
//               two-stage shared-memory ring while the previous one is
//               filtered (packed pairs again); demodulation into num / den
//               registers, carried between chunks of terms as an FP32
//               (num, den) partial;
//   k_sep_final num / den + value_range / 2 with the denominator guard.
//
// Every FIR sums its taps in increasing input order starting from zero (each
// lane of a packed multiply-add rounds like fmaf), and every demodulation step
// is the same FMA sequence as the fused kernels', so the results equal the
// fused kernels' bit for bit (zero taps, where the blocks are aligned
// differently, add exact zeros).
#include "bf_fir32.cuh"

namespace bf {

namespace {

constexpr int kSepMaxRp = 64;
struct TapsL {
    float2 g[8 * (kSepMaxRp / 4 + 1) + 16];  // (g, g), g[t + 8] = g(t - Rp), 0 outside |t - Rp| <= R
};

constexpr int kRowsR = 8;       // image rows per row-pass CTA
constexpr int kRowsW = 128;     // output columns per row-pass CTA
constexpr int kRowsNT = 256;
constexpr int kColsH = 128;     // output rows per column-pass CTA
constexpr int kColsW = 32;      // output columns per column-pass CTA
constexpr int kColsNT = 512;    // 16 warps: warp w -> rows 8w..8w+7, lane -> column

__device__ __forceinline__ int sep_terms(const SetHdr& hd) { return hd.F < 0 ? 0 : hd.F + hd.z; }

__device__ __forceinline__ void term_phase(const SepArgs& a, const SetHdr& hd, int k, float& om_hi,
                                           float& om_lo, float& Wk)
{
    om_hi = om_lo = 0.f;
    Wk = hd.w0;                 // the zero frequency (k == F): omega = 0
    if (k < hd.F) {
        const Pair p = a.pairs[k];
        om_hi = p.om_hi;
        om_lo = p.om_lo;
        Wk = p.W;
    }
}

// acc[i] += g(d - Rp) v[j], d = s0 + j - i in [0, 2 Rp] (s0 a constant after unrolling).
template <int Rp>
__device__ __forceinline__ void fir8_x2(float2 (&acc)[8], const TapsL& tp, int s0, const float2 (&v)[8])
{
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int d = s0 + j - i;
            if (d < 0 || d > 2 * Rp) continue;
            acc[i] = __ffma2_rn(tp.g[d + 8], v[j], acc[i]);
        }
}

// One 8-output FIR block of a pair from 8 * NCH input pairs starting at
// in[0] (16-byte aligned), m (may be null) multiplying each input pair.
template <int NCH>
__device__ __forceinline__ void fir_block_x2(const TapsL& tp, const float2* in, const float* m,
                                             float2 (&acc)[8])
{
    constexpr int Rp = (NCH - 1) * 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        const int a0 = ch * 8;
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 w = *(const float4*)(in + a0 + 2 * q);
            v[2 * q] = make_float2(w.x, w.y);
            v[2 * q + 1] = make_float2(w.z, w.w);
        }
        if (m) {
            const float4 f0 = *(const float4*)(m + a0), f1 = *(const float4*)(m + a0 + 4);
            const float mm[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __fmul2_rn(make_float2(mm[j], mm[j]), v[j]);
        }
        fir8_x2<Rp>(acc, tp, a0, v);
    }
}

// Row pass.  Shared memory: centred f (row pitch RW + 4 floats) and the
// (cos, sin) pairs (row pitch RW + 2 float2, an odd number of 16-byte
// chunks); a quarter-warp takes the 8 rows of one 8-column block, so its
// vector loads fall on 8 different bank groups.
template <int NCH>
__global__ void __launch_bounds__(kRowsNT)
k_sep_rows(SepArgs a, const __grid_constant__ TapsL tp, int k0)
{
    constexpr int Rp = (NCH - 1) * 4;
    constexpr int RW = kRowsW + 2 * Rp;          // halo'd columns
    constexpr int FP = RW + 4;                   // f row pitch (floats)
    constexpr int CSp = RW + 2;                  // (cos, sin) row pitch (pairs)
    static_assert((FP / 4) % 2 == 1 && (CSp / 2) % 2 == 1 && kRowsR == 8, "bank layout");
    extern __shared__ __align__(16) float sm[];
    float2* cs = (float2*)sm;                    // kRowsR x CSp
    float* fsm = sm + 2 * kRowsR * CSp;          // kRowsR x FP
    const SetHdr hd = a.hdr[0];
    const int nterms = sep_terms(hd);
    if (k0 >= nterms) return;
    const int nk = min(a.nk, nterms - k0);
    const int tid = threadIdx.x;
    const int y0 = blockIdx.y * kRowsR, xt = blockIdx.x * kRowsW, gx0 = xt - Rp;

    for (int i = tid; i < kRowsR * RW; i += kRowsNT) {
        const int r = i / RW, col = i - r * RW;
        const int gy = y0 + r, x = gx0 + col;
        float v = 0.f;
        if (gy < a.H && x >= 0 && x < a.W) v = __ldg(a.f + (size_t)gy * a.f_pitch + x) - a.c0;
        fsm[r * FP + col] = v;
    }
    __syncthreads();
    for (int kk = 0; kk < nk; ++kk) {
        float om_hi, om_lo, Wk;
        term_phase(a, hd, k0 + kk, om_hi, om_lo, Wk);
        for (int i = tid; i < kRowsR * RW; i += kRowsNT) {
            const int r = i / RW, col = i - r * RW;
            const int gy = y0 + r, x = gx0 + col;
            float c = 0.f, sn = 0.f;
            if (gy < a.H && x >= 0 && x < a.W) fir32::phase_cs(fsm[r * FP + col], om_hi, om_lo, c, sn);
            cs[r * CSp + col] = make_float2(c, sn);
        }
        __syncthreads();
        // items (pair h, block cb, row r): consecutive threads -> consecutive rows
        for (int it = tid; it < 2 * kRowsR * (kRowsW / 8); it += kRowsNT) {
            const int r = it % kRowsR, cb = (it / kRowsR) % (kRowsW / 8);
            const int h = it / (kRowsR * (kRowsW / 8));
            const int gy = y0 + r;
            float2 acc[8];
            fir_block_x2<NCH>(tp, cs + r * CSp + cb * 8, h == 0 ? fsm + r * FP + cb * 8 : nullptr, acc);
            if (gy < a.H) {
                float2* dst = a.P + (((size_t)kk * 2 + h) * a.H + gy) * a.Wp + xt + cb * 8;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *(float4*)(dst + 2 * q) =
                        make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y);
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void cp_async16z(float* dst, const float* src, bool pred)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "r"(pred ? 16 : 0)
                 : "memory");
}

template <int NCH>
__global__ void __launch_bounds__(kColsNT)
k_sep_cols(SepArgs a, const __grid_constant__ TapsL tp, int k0)
{
    constexpr int Rp = (NCH - 1) * 4;
    constexpr int RHt = kColsH + 2 * Rp;              // halo'd rows of a strip
    constexpr int kStage = RHt * kColsW;              // pairs: one strip
    extern __shared__ __align__(16) float sm[];       // two stages
    float2* sp = (float2*)sm;
    const SetHdr hd = a.hdr[0];
    const int nterms = sep_terms(hd);
    if (k0 >= nterms) return;
    const int nk = min(a.nk, nterms - k0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int by = blockIdx.y * kColsH, bx = blockIdx.x * kColsW;
    const int o = lane, rb = warp;
    const int gx = bx + o;

    // stage s of the sequence (term kk = s / 2, pair h = s % 2): strip rows
    // by - Rp .. by + 127 + Rp of that pair, 16 bytes (two pairs) per copy
    auto fetch = [&](int s) {
        float2* dst = sp + (s & 1) * kStage;
        const int kk = s >> 1, h = s & 1;
        for (int i = tid; i < RHt * (kColsW / 2); i += kColsNT) {
            const int q = i % (kColsW / 2), r = i / (kColsW / 2);
            const int gy = by - Rp + r;
            const bool ok = gy >= 0 && gy < a.H;
            const float2* src = a.P + (((size_t)kk * 2 + h) * a.H + (ok ? gy : 0)) * a.Wp + bx + 2 * q;
            cp_async16z((float*)(dst + r * kColsW + 2 * q), (const float*)src, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    float num[8], den[8];
    const bool carry = k0 > 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        num[i] = den[i] = 0.f;
        const int gy = by + rb * 8 + i;
        if (carry && gy < a.H && gx < a.W) {
            const float2 t = a.nd[(size_t)gy * a.W + gx];
            num[i] = t.x;
            den[i] = t.y;
        }
    }
    // centred f of my outputs, for the demodulation phases
    float fo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gy = by + rb * 8 + i;
        fo[i] = (gy < a.H && gx < a.W) ? __ldg(a.f + (size_t)gy * a.f_pitch + gx) - a.c0 : 0.f;
    }

    const int nst = 2 * nk;
    fetch(0);
    float2 nab[8];
    for (int s = 0; s < nst; ++s) {
        if (s + 1 < nst) fetch(s + 1);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        const float2* st = sp + (s & 1) * kStage;
        float2 acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            const int a0 = ch * 8;
            float2 v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = st[(rb * 8 + a0 + j) * kColsW + o];
            fir8_x2<Rp>(acc, tp, a0, v);
        }
        if ((s & 1) == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) nab[i] = acc[i];
        } else {
            float om_hi, om_lo, Wk;
            term_phase(a, hd, k0 + (s >> 1), om_hi, om_lo, Wk);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float c, sn;
                fir32::phase_cs(fo[i], om_hi, om_lo, c, sn);
                if (!(by + rb * 8 + i < a.H && gx < a.W)) c = sn = 0.f;
                num[i] = fmaf(Wk, fmaf(c, nab[i].x, sn * nab[i].y), num[i]);
                den[i] = fmaf(Wk, fmaf(c, acc[i].x, sn * acc[i].y), den[i]);
            }
        }
        __syncthreads();                               // stage s & 1 is refilled next
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gy = by + rb * 8 + i;
        if (gy < a.H && gx < a.W) a.nd[(size_t)gy * a.W + gx] = make_float2(num[i], den[i]);
    }
}

__global__ void k_sep_final(SepArgs a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.W) return;
    const SetHdr hd = a.hdr[0];
    const int R = a.R;
    const float full = full_mass(a.taps, R);
    const float cmass = clipped_mass(a.taps, R, x, a.W, full);
    for (int y = blockIdx.y; y < a.H; y += gridDim.y) {
        const float fv = a.f[(size_t)y * a.f_pitch + x];
        float v;
        float den = 0.f;
        if (hd.F < 0) {
            v = fv;                                  // order above the cap: pass through
        } else {
            const float rmass = clipped_mass(a.taps, R, y, a.H, full);
            const float2 nd = a.nd[(size_t)y * a.W + x];
            den = nd.y;
            if (a.fix_list && nd.y < a.fix_kappa * rmass * cmass) {
                // den a small part of the mass: the FP32 recheck writes it
                v = fv;
                a.fix_list[atomicAdd(a.fix_count, 1u)] = (unsigned)y * (unsigned)a.W + (unsigned)x;
            } else if (nd.y > kGuard * rmass * cmass) {
                v = __fdiv_rn(nd.x, nd.y) + a.c0;
            } else {
                v = fv;
                atomicAdd(a.n_guarded, 1ull);
            }
        }
        a.out[(size_t)y * a.out_pitch + x] = v;
        if (a.den_out) a.den_out[(size_t)y * a.den_pitch + x] = den;
    }
}

template <int NCH>
cudaError_t launch_nch(const SepArgs& a, const TapsL& tp, int n_chunks, cudaStream_t s)
{
    constexpr int Rp = (NCH - 1) * 4;
    constexpr int RW = kRowsW + 2 * Rp;
    const size_t smem_rows = (size_t)kRowsR * (2 * (RW + 2) + RW + 4) * sizeof(float);
    const size_t smem_cols = (size_t)2 * (kColsH + 2 * Rp) * kColsW * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_sep_rows<NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_rows);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_sep_cols<NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_cols);
    if (e != cudaSuccess) return e;
    const dim3 grow(a.Wp / kRowsW, (a.H + kRowsR - 1) / kRowsR);
    const dim3 gcol((a.W + kColsW - 1) / kColsW, (a.H + kColsH - 1) / kColsH);
    for (int c = 0; c < n_chunks; ++c) {
        k_sep_rows<NCH><<<grow, kRowsNT, smem_rows, s>>>(a, tp, c * a.nk);
        k_sep_cols<NCH><<<gcol, kColsNT, smem_cols, s>>>(a, tp, c * a.nk);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_sep_final<<<dim3((a.W + 255) / 256, a.H < 65535 ? a.H : 65535), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Radii the two-pass path takes: beyond the fused tall tile, up to Rp = 64.
bool sep32_ok(int R) { return R > 24 && (R + 3) / 4 * 4 <= kSepMaxRp; }

int sep32_width(int W) { return (W + kRowsW - 1) / kRowsW * kRowsW; }

cudaError_t launch_sep32(const SepArgs& a, int n_terms_cap, cudaStream_t s)
{
    if (!sep32_ok(a.R) || !a.h_taps || a.nk < 1) return cudaErrorInvalidValue;
    const int Rp = (a.R + 3) / 4 * 4;
    TapsL tp;
    for (int i = 0; i < (int)(sizeof(tp.g) / sizeof(float2)); ++i) {
        const int k = i - 8 - Rp;
        const float g = (k >= -a.R && k <= a.R) ? a.h_taps[k + a.R] : 0.f;
        tp.g[i] = make_float2(g, g);
    }
    const int n_chunks = (n_terms_cap + a.nk - 1) / a.nk;
    switch (Rp / 4 + 1) {
    case 8: return launch_nch<8>(a, tp, n_chunks, s);
    case 9: return launch_nch<9>(a, tp, n_chunks, s);
    case 10: return launch_nch<10>(a, tp, n_chunks, s);
    case 11: return launch_nch<11>(a, tp, n_chunks, s);
    case 12: return launch_nch<12>(a, tp, n_chunks, s);
    case 13: return launch_nch<13>(a, tp, n_chunks, s);
    case 14: return launch_nch<14>(a, tp, n_chunks, s);
    case 15: return launch_nch<15>(a, tp, n_chunks, s);
    case 16: return launch_nch<16>(a, tp, n_chunks, s);
    case 17: return launch_nch<17>(a, tp, n_chunks, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bf
