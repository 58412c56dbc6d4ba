// K3: fused SHIFTABLE-BF forward with FP32 planes and an exact FIR Gaussian.
//
// Sec. 1.2 of the paper (eqs. (f1), (f2) and the four-step procedure): for
// each kept term of phi_eps (eq. (approx)) form the planes f cos(w f),
// f sin(w f), cos(w f), sin(w f), filter them with the spatial Gaussian
// (eq. (GF)), demodulate with cos(w f(x)), sin(w f(x)) and accumulate the
// numerator and the denominator; out = num / den.  Terms n and N-n are folded
// (cos is even: their contributions are equal), so a pair carries 2 w_n.
//
// GB300 form, one CTA per TH x TW block of outputs, one launch per image:
//   * the block plus its R halo of the centred image f - c0 is staged in
//     shared memory once; HBM sees f once and out once;
//   * per pair: (1) every halo pixel gets cos / sin of its phase, computed as
//     an FP32 head + tail product (FMA TwoProduct) reduced by 2 pi in two
//     parts (Cody-Waite) and evaluated on the SFU; (2) rows are filtered with
//     a register-blocked FIR (8 outputs per thread, 8 inputs per step, taps
//     zero-padded so that no branch guards the window); (3) columns likewise,
//     then the demodulation FMAs go straight into num / den registers;
//   * out-of-image pixels have all four planes zero (clipped windows);
//   * a pixel whose den <= 1e-6 (g * 1_Omega) keeps f (the paper is silent).
#include <math.h>

#include "bf_fir32.cuh"

namespace bf {
namespace {

using fir32::Geo;
using fir32::phase_cs;

// One output tile with origin (by, bx): the whole block takes part.
template <int TH, int TW>
__device__ __forceinline__ void fwd32_body(const FwdArgs& a, int by, int bx, float* sm)
{
    constexpr int NT = TH * TW / 8;
    constexpr int NW = NT / 32;
    const Geo G(a.R, TH, TW);
    const int R = a.R;
    float* fsm = sm;                              // RH x RWp  centred f, 0 outside
    float* csm = fsm + (size_t)G.RH * G.RWp;      // RH x RWp  cos
    float* ssm = csm + (size_t)G.RH * G.RWp;      // RH x RWp  sin
    float* hsm = ssm + (size_t)G.RH * G.RWp;      // 4 x RHp x TW  row-filtered planes
    float* gz = hsm + 4 * (size_t)G.RHp * TW;     // taps, gz[t + 8] = g(t - R), 0 outside [0, 2R]
    const size_t hplane = (size_t)G.RHp * TW;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gy0 = by - R, gx0 = bx - R;

    const int set = a.set_tile ? (by / a.set_tile) * a.sets_x + (bx / a.set_tile) : 0;
    const SetHdr hd = a.hdr[set];

    // my vertical item: column o, rows rb*8 .. rb*8+7 of the block
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

    // stage the centred block + halo (and zero the padding columns)
    for (int r = warp; r < G.RH; r += NW) {
        const int gy = gy0 + r;
        const bool rin = gy >= 0 && gy < a.H;
        for (int col = lane; col < G.RWp; col += 32) {
            const int x = gx0 + col;
            float v = 0.f;
            if (rin && col < G.RW && x >= 0 && x < a.W)
                v = __ldg(a.f + (size_t)gy * a.f_pitch + x) - a.c0;
            fsm[r * G.RWp + col] = v;
        }
    }
    for (int i = tid; i < G.ngz; i += NT) {
        const int t = i - 8;
        gz[i] = (t >= 0 && t <= 2 * R) ? a.taps[t] : 0.f;
    }
    // rows RH..RHp-1 of the row-filtered planes stay zero for the whole launch
    for (int i = tid; i < (G.RHp - G.RH) * TW; i += NT)
        for (int q = 0; q < 4; ++q) hsm[q * hplane + (size_t)G.RH * TW + i] = 0.f;

    // clipped Gaussian mass of my outputs (denominator guard)
    const float full = full_mass(a.taps, R);
    const float cmass = clipped_mass(a.taps, R, gx, a.W, full);

    float num[8], den[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) num[i] = den[i] = 0.f;

    __syncthreads();

    const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    const int K = hd.F + hd.z;
    for (int k = 0; k < K; ++k) {
        float om_hi = 0.f, om_lo = 0.f, Wk = hd.w0;
        if (k < hd.F) {
            const Pair p = pr[k];
            om_hi = p.om_hi;
            om_lo = p.om_lo;
            Wk = p.W;
        }

        // (1) modulate: cos / sin of every in-image halo pixel, 0 elsewhere
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

        // (2) rows: item (r, cb) -> 8 outputs of row r, columns cb*8 .. cb*8+7
        fir32::row_pass<TW, true>(G, fsm, nullptr, csm, ssm, gz, hsm, tid, NT);
        __syncthreads();

        // (3) columns of my item, then demodulate into num / den
        {
            float acc[4][8];
            fir32::col_pass<TW>(G, hsm, gz, o, rb, acc);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int ry = rb * 8 + i + R;
                const float c = csm[ry * G.RWp + o + R], s = ssm[ry * G.RWp + o + R];
                num[i] = fmaf(Wk, fmaf(c, acc[0][i], s * acc[1][i]), num[i]);
                den[i] = fmaf(Wk, fmaf(c, acc[2][i], s * acc[3][i]), den[i]);
            }
        }
        __syncthreads();
    }

    // normalise (eq. (f1) over eq. (f2)) with the guard, write out; outputs
    // whose den is under fix_kappa of their mass are listed for the FP32
    // recheck (large windows: the FP32 rounding of the planes is amplified by
    // mass / den there), which writes them
    if (gx < a.W) {
        const float kap = a.fix_list ? a.fix_kappa : -INFINITY;
        uint32_t listed = 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gy = by + rb * 8 + i;
            if (gy >= a.H) continue;
            const float rmass = clipped_mass(a.taps, R, gy, a.H, full);
            float v;
            if (den[i] < kap * rmass * cmass) {
                listed |= 1u << i;
                v = a.f[(size_t)gy * a.f_pitch + gx];
            } else if (den[i] > kGuard * rmass * cmass) {
                v = __fdiv_rn(num[i], den[i]) + a.c0;
            } else {
                v = a.f[(size_t)gy * a.f_pitch + gx];
                atomicAdd(a.n_guarded, 1ull);
            }
            a.out[(size_t)gy * a.out_pitch + gx] = v;
            if (a.den_out) a.den_out[(size_t)gy * a.den_pitch + gx] = den[i];
        }
        while (listed) {
            const int i = __ffs(listed) - 1;
            listed &= listed - 1u;
            a.fix_list[(size_t)set * a.fix_cap + atomicAdd(a.fix_count + set, 1u)] =
                (unsigned)(by + rb * 8 + i) * (unsigned)a.W + (unsigned)gx;
        }
    }
}

// Tall-tile form (128 x 32 outputs, 512 threads): the cos and sin planes of
// a pass are filtered together as packed pairs (see TallGeo).  Same
// arithmetic per output as fwd32_body: each lane of a packed multiply-add
// rounds like fmaf, the nonzero taps are summed in the same order and the
// skipped ones would have added exact zeros.
//
// NCH = Rp / 4 + 1 is a template parameter and the taps arrive as kernel
// parameters (tp.g[t + 8] = g(t - Rp), tp2 the same as pairs), so the fully
// unrolled FIR takes every tap from the constant bank; the taps are the
// plan's FP32 taps, the same words the shared-memory form reads.
//
// Per pair k: row pass of (f' c, f' s) -> column pass -> numerator; row pass
// of (c, s) -> column pass -> denominator.  The last column pass reads only
// the row-filtered buffer, so the phases of pair k + 1 are written into cs
// during it, their independent SFU / FMA chains filling the issue slots the
// packed multiply-adds leave free; the denominator's demodulation then takes
// cos / sin of pair k at its own outputs from the same phase function.
template <int TH, int TW, int NCH, bool kBox>
__device__ __forceinline__ void fwd32t_body(const FwdArgs& a, const fir32::Taps& tp,
                                            const fir32::Taps2& tp2, int by, int bx, char* sm)
{
    using G = fir32::TallGeo<TH, TW, NCH>;
    constexpr int CO = 8;                      // a thread owns CO outputs of one column
    constexpr int NT = TH * TW / CO;
    constexpr int Rp = G::Rp;
    constexpr int NPX = G::RH * G::RW;         // halo pixels
    static_assert(NT / G::RW >= 1, "phase sweep");
    constexpr int NS = CO / 8 + NCH - 1;       // input steps of the column pass
    using PS = fir32::PhaseSweep<G, NT>;
    constexpr int PPS = (PS::ITERS + NS - 1) / NS;               // phase rows per column step
    float2* cs = (float2*)sm;                                   // RH x CSp (cos, sin)
    float* fz = (float*)(sm + G::cs_bytes);                     // RH x FP  centred f
    float2* hz = (float2*)(sm + G::cs_bytes + G::fz_bytes);     // RH x TW  row-filtered pair

    const int tid = threadIdx.x;
    const int gy0 = by - Rp, gx0 = bx - Rp;
    const int set = a.set_tile ? (by / a.set_tile) * a.sets_x + (bx / a.set_tile) : 0;
    const SetHdr hd = a.hdr[set];
    const int o = tid % TW, rb = tid / TW;
    const int gx = bx + o;

    if (hd.F < 0) {          // order above the cap: pass the image through
        for (int i = 0; i < CO; ++i) {
            const int gy = by + rb * CO + i;
            if (gy < a.H && gx < a.W)
                a.out[(size_t)gy * a.out_pitch + gx] = a.f[(size_t)gy * a.f_pitch + gx];
        }
        return;
    }
    for (int e = tid; e < NPX; e += NT) {
        const int r = e / G::RW, col = e - r * G::RW;
        const int gy = gy0 + r, x = gx0 + col;
        float v = 0.f;
        if (gy >= 0 && gy < a.H && x >= 0 && x < a.W)
            v = __ldg(a.f + (size_t)gy * a.f_pitch + x) - a.c0;
        fz[r * G::FP + col] = v;
    }
    const int R = a.R;
    const float* taps = tp.g + Rp + 8 - R;          // taps[t + R] = g(t)
    const float full = full_mass(taps, R);
    const float cmass = clipped_mass(taps, R, gx, a.W, full);
    float num[CO], den[CO];
#pragma unroll
    for (int i = 0; i < CO; ++i) num[i] = den[i] = 0.f;

    const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    const int K = hd.F + hd.z;
    // frequency and weight of pair k (the zero-frequency term last)
    auto pair_of = [&](int k, float& om_hi, float& om_lo, float& Wk) {
        om_hi = 0.f;
        om_lo = 0.f;
        Wk = hd.w0;
        if (k < hd.F) {
            const Pair p = pr[k];
            om_hi = p.om_hi;
            om_lo = p.om_lo;
            Wk = p.W;
        }
    };
    float om_hi, om_lo, Wk;
    pair_of(0, om_hi, om_lo, Wk);
    const PS ps(tid, gy0, gx0, a.W);
    __syncthreads();
    fir32::PhaseSteps<PS, 0, PS::ITERS>::run(ps, fz, cs, a.H, om_hi, om_lo);
    __syncthreads();

    // sweep row m of this thread is in the halo (the last row block may overhang)
    auto sweep_row = [&](int m) {
        return ps.on && (m < PS::ITERS - 1 || ps.r0 + PS::S * m < G::RH);
    };
    // column pass of the row-filtered pair with job(m), m = ch * PPS + u, run
    // between its input steps
    auto col_pass_with = [&](float2 (&acc)[CO], auto&& job) {
        if constexpr (kBox) {
            // box: the FIR sum for the first output, sliding sums for the rest
            // (as the row pass's row_item_box_x2)
            float2 sb = make_float2(0.f, 0.f);
#pragma unroll
            for (int ch = 0; ch < NS; ++ch) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (ch * 8 + j <= 2 * Rp)
                        sb = __ffma2_rn(tp2.g[ch * 8 + j + 8],
                                        hz[fir32::hz_at(rb * CO + ch * 8 + j, o)], sb);
#pragma unroll
                for (int u = 0; u < PPS; ++u)
                    if (ch * PPS + u < PS::ITERS) job(ch * PPS + u);
            }
            acc[0] = sb;
#pragma unroll
            for (int i = 1; i < CO; ++i) {
                sb = __fadd2_rn(sb, hz[fir32::hz_at(rb * CO + i + Rp + R, o)]);
                sb = __ffma2_rn(make_float2(-1.f, -1.f), hz[fir32::hz_at(rb * CO + i - 1 + Rp - R, o)],
                                sb);
                acc[i] = sb;
            }
        } else {
#pragma unroll
            for (int i = 0; i < CO; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
            for (int ch = 0; ch < NS; ++ch) {
                float2 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = hz[fir32::hz_at(rb * CO + ch * 8 + j, o)];
                fir32::fir_x2<CO, 8, Rp>(acc, tp2, ch * 8, v);
#pragma unroll
                for (int u = 0; u < PPS; ++u)
                    if (ch * PPS + u < PS::ITERS) job(ch * PPS + u);
            }
        }
    };

    for (int k = 0; k < K; ++k) {
        // denominator pair (c, s); cos / sin at my outputs kept for both
        // demodulations, read before cs is rescaled
        fir32::row_pass_x2<TH, TW, NCH, NT, kBox>(tp2, cs, hz, tid, R);
        float2 cc[CO];
#pragma unroll
        for (int i = 0; i < CO; ++i) cc[i] = cs[(rb * CO + i + Rp) * G::CSp + o + Rp];
        __syncthreads();
        {
            // during the column pass: (c, s) -> (f'c, f's) in place, once per pixel
            float2 dcd[CO];
            col_pass_with(dcd, [&](int m) {
                if (sweep_row(m)) {
                    const int ci = ps.cbase + PS::S * m * G::CSp;
                    const float fv = fz[ps.fbase + PS::S * m * G::FP];
                    cs[ci] = __fmul2_rn(make_float2(fv, fv), cs[ci]);
                }
            });
#pragma unroll
            for (int i = 0; i < CO; ++i)
                den[i] = fmaf(Wk, fmaf(cc[i].x, dcd[i].x, cc[i].y * dcd[i].y), den[i]);
        }
        __syncthreads();
        // numerator pair (f'c, f's), already formed
        fir32::row_pass_x2<TH, TW, NCH, NT, kBox>(tp2, cs, hz, tid, R);
        __syncthreads();
        {
            // during the column pass: the phases of pair k + 1 into cs
            const bool next = k + 1 < K;
            float nx_hi, nx_lo, nW;
            pair_of(k + 1, nx_hi, nx_lo, nW);
            float2 nab[CO];
            col_pass_with(nab, [&](int m) {
                if (next && sweep_row(m)) {
                    float c, sn;
                    phase_cs(fz[ps.fbase + PS::S * m * G::FP], nx_hi, nx_lo, c, sn);
                    const bool in = ps.x_in && (unsigned)(ps.gyb + PS::S * m) < (unsigned)a.H;
                    cs[ps.cbase + PS::S * m * G::CSp] = in ? make_float2(c, sn) : make_float2(0.f, 0.f);
                }
            });
#pragma unroll
            for (int i = 0; i < CO; ++i)
                num[i] = fmaf(Wk, fmaf(cc[i].x, nab[i].x, cc[i].y * nab[i].y), num[i]);
            om_hi = nx_hi;
            om_lo = nx_lo;
            Wk = nW;
        }
        __syncthreads();
    }
    if (gx < a.W) {
#pragma unroll
        for (int i = 0; i < CO; ++i) {
            const int gy = by + rb * CO + i;
            if (gy >= a.H) continue;
            const float rmass = clipped_mass(taps, R, gy, a.H, full);
            float v;
            if (den[i] > kGuard * rmass * cmass) {
                v = __fdiv_rn(num[i], den[i]) + a.c0;
            } else {
                v = a.f[(size_t)gy * a.f_pitch + gx];
                atomicAdd(a.n_guarded, 1ull);
            }
            a.out[(size_t)gy * a.out_pitch + gx] = v;
            if (a.den_out) a.den_out[(size_t)gy * a.den_pitch + gx] = den[i];
        }
    }
}

template <int TH, int TW, int NCH, bool kBox>
__global__ void __launch_bounds__(TH * TW / 8, 1)
k_fwd32t(FwdArgs a, const __grid_constant__ fir32::Taps tp, const __grid_constant__ fir32::Taps2 tp2)
{
    extern __shared__ __align__(16) char smc[];
    fwd32t_body<TH, TW, NCH, kBox>(a, tp, tp2, blockIdx.y * TH, blockIdx.x * TW, smc);
}

template <int TH, int NCH, bool kBox>
cudaError_t launch_tall_th(const FwdArgs& a, const fir32::Taps& tp, const fir32::Taps2& tp2,
                           cudaStream_t s)
{
    constexpr size_t smem = fir32::TallGeo<TH, 32, NCH>::bytes;
    cudaError_t e = cudaFuncSetAttribute(k_fwd32t<TH, 32, NCH, kBox>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + 31) / 32, (a.H + TH - 1) / TH);
    k_fwd32t<TH, 32, NCH, kBox><<<grid, TH * 4, smem, s>>>(a, tp, tp2);
    return cudaGetLastError();
}

// 128-row tiles, or 64-row tiles where the T-tiles are 64 (not 128) rows
// high; the box spatial filter takes the sliding-sum form.
template <int NCH>
cudaError_t launch_tall(const FwdArgs& a, const fir32::Taps& tp, const fir32::Taps2& tp2,
                        cudaStream_t s)
{
    const bool th64 = fwd32t_rows(a.set_tile) == 64;
    if (a.box) return th64 ? launch_tall_th<64, NCH, true>(a, tp, tp2, s)
                           : launch_tall_th<128, NCH, true>(a, tp, tp2, s);
    return th64 ? launch_tall_th<64, NCH, false>(a, tp, tp2, s)
                : launch_tall_th<128, NCH, false>(a, tp, tp2, s);
}

template <int TH, int TW>
__global__ void __launch_bounds__(TH * TW / 8, 1) k_fwd32(FwdArgs a)
{
    extern __shared__ __align__(16) float sm[];
    fwd32_body<TH, TW>(a, blockIdx.y * TH, blockIdx.x * TW, sm);
}

// Persistent form: CTAs take (image, tile) items from a queue (atomic head)
// until it is empty; items are ordered by the caller (costly first).
template <int TH, int TW>
__global__ void __launch_bounds__(TH * TW / 8, 1)
k_fwd32_persistent(const FwdArgs* __restrict__ imgs, const int4* __restrict__ items, int n_items,
                   unsigned* __restrict__ head)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();                       // the previous item is done with shared memory
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int i = s_item;
        if (i >= n_items) break;
        const int4 it = items[i];              // (image, tile row origin, tile column origin, -)
        const FwdArgs a = imgs[it.x];
        fwd32_body<TH, TW>(a, it.y, it.z, sm);
    }
}

template <int TH, int TW>
cudaError_t launch_tile(const FwdArgs& a, cudaStream_t s)
{
    const Geo G(a.R, TH, TW);
    const size_t smem = G.floats(TW, 3) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_fwd32<TH, TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    k_fwd32<TH, TW><<<grid, TH * TW / 8, smem, s>>>(a);
    return cudaGetLastError();
}

constexpr size_t kSmemLimit = 227 * 1024;

}  // namespace

size_t fwd32_smem(int R, int th, int tw)
{
    return Geo(R, th, tw).floats(tw, 3) * sizeof(float);
}

void fwd32_tile(int R, int* th, int* tw)
{
    static const int shapes[][2] = {{64, 32}, {32, 32}, {16, 16}};
    for (auto& sh : shapes)
        if (fwd32_smem(R, sh[0], sh[1]) <= kSmemLimit) {
            *th = sh[0];
            *tw = sh[1];
            return;
        }
    *th = *tw = 0;
}

int fwd32_persistent_ctas_per_sm(int th, int tw, int max_R)
{
    const size_t smem = fwd32_smem(max_R, th, tw);
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define BF_OCC(TH_, TW_)                                                                  \
    if (th == TH_ && tw == TW_) {                                                         \
        e = cudaFuncSetAttribute(k_fwd32_persistent<TH_, TW_>,                            \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e == cudaSuccess)                                                             \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                            \
                &n, k_fwd32_persistent<TH_, TW_>, TH_ * TW_ / 8, smem);                   \
    }
    BF_OCC(64, 32)
    BF_OCC(32, 32)
    BF_OCC(16, 16)
#undef BF_OCC
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_fwd32_persistent(int th, int tw, int max_R, const FwdArgs* imgs,
                                   const int4* items, int n_items, unsigned* head, int n_ctas,
                                   cudaStream_t s)
{
    const size_t smem = fwd32_smem(max_R, th, tw);
    cudaError_t e = cudaErrorInvalidValue;
#define BF_PERSIST(TH_, TW_)                                                               \
    if (th == TH_ && tw == TW_) {                                                          \
        e = cudaFuncSetAttribute(k_fwd32_persistent<TH_, TW_>,                             \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
        if (e != cudaSuccess) return e;                                                    \
        k_fwd32_persistent<TH_, TW_><<<n_ctas, TH_ * TW_ / 8, smem, s>>>(imgs, items,      \
                                                                           n_items, head); \
        return cudaGetLastError();                                                         \
    }
    BF_PERSIST(64, 32)
    BF_PERSIST(32, 32)
    BF_PERSIST(16, 16)
#undef BF_PERSIST
    return e;
}

// Output rows of the tall tile for T-tiles of set_tile rows (0: one set):
// the tile must nest inside a T-tile.
int fwd32t_rows(int set_tile)
{
    if (set_tile == 0 || set_tile % 128 == 0) return 128;
    if (set_tile % 64 == 0) return 64;
    return 0;
}

size_t fwd32t_smem(int R, int rows)
{
#define BF_TALL_SMEM(N_)                                                                 \
    case N_: return rows == 64 ? fir32::TallGeo<64, 32, N_>::bytes : fir32::TallGeo<128, 32, N_>::bytes;
    switch ((R + 3) / 4 + 1) {
        BF_TALL_SMEM(2)
        BF_TALL_SMEM(3)
        BF_TALL_SMEM(4)
        BF_TALL_SMEM(5)
        BF_TALL_SMEM(6)
        BF_TALL_SMEM(7)
        default: return (size_t)-1;
    }
#undef BF_TALL_SMEM
}

// The tall tile serves a launch when its padded radius has a compiled tap
// count, its shared memory fits and its tiles nest inside the T-tiles.
bool fwd32t_ok(int R, int set_tile)
{
    const int rows = fwd32t_rows(set_tile);
    return R >= 1 && (R + 3) / 4 * 4 <= fir32::kTapsMaxRp && rows > 0 &&
           fwd32t_smem(R, rows) <= kSmemLimit;
}

cudaError_t launch_fwd32(const FwdArgs& a, cudaStream_t s)
{
    if (a.box_rs) return launch_box32(a, s);     // box filter: exact running sums
    if (a.sep_P && a.set_tile == 0 && !fwd32t_ok(a.R, 0) && sep32_ok(a.R)) {
        SepArgs sa;
        sa.f = a.f;
        sa.f_pitch = a.f_pitch;
        sa.out = a.out;
        sa.out_pitch = a.out_pitch;
        sa.H = a.H;
        sa.W = a.W;
        sa.Wp = a.sep_Wp;
        sa.R = a.R;
        sa.c0 = a.c0;
        sa.hdr = a.hdr;
        sa.pairs = a.pairs;
        sa.taps = a.taps;
        sa.h_taps = a.h_taps;
        sa.P = reinterpret_cast<float2*>(a.sep_P);
        sa.nd = a.sep_nd;
        sa.nk = a.sep_nk;
        sa.n_guarded = a.n_guarded;
        sa.den_out = a.den_out;
        sa.den_pitch = a.den_pitch;
        sa.fix_list = a.fix_list;
        sa.fix_count = a.fix_count;
        sa.fix_kappa = a.fix_kappa;
        return launch_sep32(sa, a.sep_cap_terms, s);
    }
    if (a.h_taps && fwd32t_ok(a.R, a.set_tile)) {
        const int Rp = (a.R + 3) / 4 * 4;
        fir32::Taps tp;
        fir32::Taps2 tp2;
        for (int i = 0; i < (int)(sizeof(tp.g) / sizeof(float)); ++i) {
            const int k = i - 8 - Rp;
            tp.g[i] = (k >= -a.R && k <= a.R) ? a.h_taps[k + a.R] : 0.f;
            tp2.g[i] = make_float2(tp.g[i], tp.g[i]);
        }
        switch (Rp / 4 + 1) {
            case 2: return launch_tall<2>(a, tp, tp2, s);
            case 3: return launch_tall<3>(a, tp, tp2, s);
            case 4: return launch_tall<4>(a, tp, tp2, s);
            case 5: return launch_tall<5>(a, tp, tp2, s);
            case 6: return launch_tall<6>(a, tp, tp2, s);
            case 7: return launch_tall<7>(a, tp, tp2, s);
            default: break;
        }
    }
    int th, tw;
    fwd32_tile(a.R, &th, &tw);
    if (th == 64 && tw == 32) return launch_tile<64, 32>(a, s);
    if (th == 32 && tw == 32) return launch_tile<32, 32>(a, s);
    if (th == 16 && tw == 16) return launch_tile<16, 16>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace bf
