// K3-sep: the FP32 FIR forward (Sec. 1.2, eqs. (f1)-(f2)) in two passes
// through HBM, for radii whose halo does not fit a fused tile (R > 24) in
// plans with one parameter set.
//
// The fused kernels keep a tile and its 2R halo in shared memory; beyond
// R = 24 only 32 x 32 or 16 x 16 tiles fit, and their halo work grows to
// 7-50 times the outputs.  Here the two separable passes meet in HBM:
//
//   k_sep_rows  a CTA takes 8 image rows x 128 output columns (+ R halo
//               columns): f once, then per term its phases and the 4 planes
//               f'c, f's, c, s filtered along the row (8 outputs x 8 inputs
//               per register-blocked step, taps as constant-bank operands),
//               written to a buffer of nk terms, [term][plane][H][Wp];
//   k_sep_cols  a CTA takes 128 x 32 outputs: per term and plane pair, the
//               (128 + 2R) x 32 column strip arrives by cp.async in a
//               two-stage shared-memory ring while the previous one is
//               filtered; demodulation into num / den registers, carried
//               between chunks of terms as an FP32 (num, den) partial;
//   k_sep_final num / den + value_range / 2 with the denominator guard.
//
// Every FIR sums its taps in increasing input order starting from zero, and
// every demodulation step is the same FMA sequence as the fused kernels', so
// the results equal the fused kernels' bit for bit (zero taps, where the
// blocks are aligned differently, add exact zeros).
#include "bf_fir32.cuh"

namespace bf {

namespace {

constexpr int kSepMaxRp = 64;
struct TapsL {
    float g[8 * (kSepMaxRp / 4 + 1) + 16];   // g[t + 8] = g(t - Rp), 0 outside |t - Rp| <= R
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

// One 8-output FIR block from 8 * NCH inputs starting at in[0] (FP32,
// 16-byte aligned), taps from tp; m (may be null) multiplies each input.
template <int NCH>
__device__ __forceinline__ void fir_block(const TapsL& tp, const float* in, const float* m,
                                          float (&acc)[8])
{
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        const int a0 = ch * 8;
        float g[15];
#pragma unroll
        for (int d = 0; d < 15; ++d) g[d] = tp.g[a0 + d + 1];
        const float4 v0 = *(const float4*)(in + a0), v1 = *(const float4*)(in + a0 + 4);
        float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        if (m) {
            const float4 f0 = *(const float4*)(m + a0), f1 = *(const float4*)(m + a0 + 4);
            v[0] *= f0.x; v[1] *= f0.y; v[2] *= f0.z; v[3] *= f0.w;
            v[4] *= f1.x; v[5] *= f1.y; v[6] *= f1.z; v[7] *= f1.w;
        }
        if (ch == 0) fir32::fir_step<1>(acc, g, v);
        else if (ch == NCH - 1) fir32::fir_step<2>(acc, g, v);
        else fir32::fir_step<0>(acc, g, v);
    }
}

template <int NCH>
__global__ void __launch_bounds__(kRowsNT)
k_sep_rows(SepArgs a, const __grid_constant__ TapsL tp, int k0)
{
    constexpr int Rp = (NCH - 1) * 4;
    constexpr int RW = kRowsW + 2 * Rp;          // halo'd columns
    constexpr int RWs = RW + 4;                  // row stride (bank stagger)
    extern __shared__ __align__(16) float sm[];
    float* fsm = sm;                             // centred f, 0 outside the image
    float* csm = fsm + kRowsR * RWs;             // cos
    float* ssm = csm + kRowsR * RWs + 4;         // sin (bank-staggered)
    const SetHdr hd = a.hdr[0];
    const int nterms = sep_terms(hd);
    if (k0 >= nterms) return;
    const int nk = min(a.nk, nterms - k0);
    const int tid = threadIdx.x;
    const int y0 = blockIdx.y * kRowsR, xt = blockIdx.x * kRowsW, gx0 = xt - Rp;

    for (int i = tid; i < kRowsR * RWs; i += kRowsNT) {
        const int r = i / RWs, col = i - r * RWs;
        const int gy = y0 + r, x = gx0 + col;
        float v = 0.f;
        if (gy < a.H && col < RW && x >= 0 && x < a.W) v = __ldg(a.f + (size_t)gy * a.f_pitch + x) - a.c0;
        fsm[i] = v;
    }
    __syncthreads();
    for (int kk = 0; kk < nk; ++kk) {
        float om_hi, om_lo, Wk;
        term_phase(a, hd, k0 + kk, om_hi, om_lo, Wk);
        for (int i = tid; i < kRowsR * RWs; i += kRowsNT) {
            const int r = i / RWs, col = i - r * RWs;
            const int gy = y0 + r, x = gx0 + col;
            float c = 0.f, s = 0.f;
            if (gy < a.H && col < RW && x >= 0 && x < a.W) fir32::phase_cs(fsm[i], om_hi, om_lo, c, s);
            csm[i] = c;
            ssm[i] = s;
        }
        __syncthreads();
        // items: (plane p, row r, block cb); consecutive threads -> consecutive cb
        for (int it = tid; it < 4 * kRowsR * (kRowsW / 8); it += kRowsNT) {
            const int cb = it % (kRowsW / 8), r = (it / (kRowsW / 8)) % kRowsR;
            const int p = it / (kRowsR * (kRowsW / 8));
            const int gy = y0 + r;
            const float* src = ((p & 1) ? ssm : csm) + r * RWs + cb * 8;
            const float* mr = p < 2 ? fsm + r * RWs + cb * 8 : nullptr;
            float acc[8];
            fir_block<NCH>(tp, src, mr, acc);
            if (gy < a.H) {
                float* dst = a.P + (((size_t)kk * 4 + p) * a.H + gy) * a.Wp + xt + cb * 8;
                *(float4*)dst = make_float4(acc[0], acc[1], acc[2], acc[3]);
                *(float4*)(dst + 4) = make_float4(acc[4], acc[5], acc[6], acc[7]);
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
    constexpr int kStage = 2 * RHt * kColsW;          // floats: two planes
    extern __shared__ __align__(16) float sm[];       // two stages
    const SetHdr hd = a.hdr[0];
    const int nterms = sep_terms(hd);
    if (k0 >= nterms) return;
    const int nk = min(a.nk, nterms - k0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int by = blockIdx.y * kColsH, bx = blockIdx.x * kColsW;
    const int o = lane, rb = warp;
    const int gx = bx + o;

    // stage s of the sequence (term kk = s / 2, plane pair h = s % 2): strip
    // rows by - Rp .. by + 127 + Rp of planes 2h, 2h + 1, 16 bytes per copy
    auto fetch = [&](int s) {
        float* dst = sm + (s & 1) * kStage;
        const int kk = s >> 1, h = s & 1;
        for (int i = tid; i < 2 * RHt * (kColsW / 4); i += kColsNT) {
            const int q = i % (kColsW / 4), r = (i / (kColsW / 4)) % RHt, pl = i / (RHt * (kColsW / 4));
            const int gy = by - Rp + r;
            const bool ok = gy >= 0 && gy < a.H;
            const float* src = a.P + (((size_t)kk * 4 + 2 * h + pl) * a.H + (ok ? gy : 0)) * a.Wp + bx + 4 * q;
            cp_async16z(dst + (pl * RHt + r) * kColsW + 4 * q, src, ok);
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
    float nab[2][8];
    for (int s = 0; s < nst; ++s) {
        if (s + 1 < nst) fetch(s + 1);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        const float* st = sm + (s & 1) * kStage;
        float acc[2][8];
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
                v0[j] = st[r * kColsW + o];
                v1[j] = st[(RHt + r) * kColsW + o];
            }
            if (ch == 0) {
                fir32::fir_step<1>(acc[0], g, v0);
                fir32::fir_step<1>(acc[1], g, v1);
            } else if (ch == NCH - 1) {
                fir32::fir_step<2>(acc[0], g, v0);
                fir32::fir_step<2>(acc[1], g, v1);
            } else {
                fir32::fir_step<0>(acc[0], g, v0);
                fir32::fir_step<0>(acc[1], g, v1);
            }
        }
        if ((s & 1) == 0) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int i = 0; i < 8; ++i) nab[q][i] = acc[q][i];
        } else {
            float om_hi, om_lo, Wk;
            term_phase(a, hd, k0 + (s >> 1), om_hi, om_lo, Wk);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float c, sn;
                fir32::phase_cs(fo[i], om_hi, om_lo, c, sn);
                if (!(by + rb * 8 + i < a.H && gx < a.W)) c = sn = 0.f;
                num[i] = fmaf(Wk, fmaf(c, nab[0][i], sn * nab[1][i]), num[i]);
                den[i] = fmaf(Wk, fmaf(c, acc[0][i], sn * acc[1][i]), den[i]);
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
            if (nd.y > kGuard * rmass * cmass) {
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
    const size_t smem_rows = (size_t)(3 * kRowsR * (kRowsW + 2 * Rp + 4) + 4) * sizeof(float);
    const size_t smem_cols = (size_t)2 * 2 * (kColsH + 2 * Rp) * kColsW * sizeof(float);
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
    for (int i = 0; i < (int)(sizeof(tp.g) / sizeof(float)); ++i) {
        const int k = i - 8 - Rp;
        tp.g[i] = (k >= -a.R && k <= a.R) ? a.h_taps[k + a.R] : 0.f;
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
