// SHIFTABLE-BF with the box spatial filter (the constant filter of Sec. 4's
// comparison with BF2) by running sums: O(1) work per plane value at any
// radius, where the FIR costs 2R + 1 multiply-adds.
//
// Per kept pair the four planes (f c, f s, c, s) (f centred and scaled by
// c0, so that every plane value of an image within [0, value_range] lies in
// [-1, 1]) are quantised to integers of 2^-21 (round to nearest; an absolute
// error of at most 2^-22, two FP32 unit roundoffs at 1), and the box sums
// are taken exactly in integer arithmetic: along each halo row a running sum
// of 2R + 1 values (int32: (2R + 1) 8 2^21 < 2^31 for R <= 63, so values up
// to 8 in magnitude are exact; larger ones, from images far outside their
// value range, are clamped there), along each column a running sum of 2R + 1
// row sums (int64).  Exact sums do not drift, so a running sum is
// as accurate as a direct one; the only roundings are the quantisation and
// the conversion of each box sum back to FP32 (2^-24 relative).  The phases,
// the demodulation (eqs. (f1), (f2)), the zero frequency, the clipped
// windows (planes are zero outside the image) and the denominator guard are
// those of the FIR kernels.
//
// One CTA of 4 TH threads per TH x 32 tile of outputs.  Per pair: the
// phases of the halo (FP32 head + exact tail, two-part 2 pi reduction, SFU
// sincos), then for the denominator's planes (c, s) and then the
// numerator's (f c, f s): row sums (one thread per halo row, plane and
// half-row: a start sum of 2R + 1 values, then one add and one subtract per
// output), column sums and demodulation (one thread per column and 8 rows,
// both planes), num / den kept in registers across the pairs.
//
// Where it serves: the library runs it for the box filter where the FIR
// would need its small 16 x 16 tiles (per-T-tile plans with R above about
// 40, whose fused FIR tiles no longer fit); measured on GB300 at 2048^2,
// sigma_r = 5, per-128^2 T-tile, R = 48: 46.8 ms against 334 ms.  At smaller
// radii the FIR with packed FP32 multiply-adds is faster (R = 20: 3.3 ms
// against 5.8 ms): with one CTA per SM (its shared memory) the running-sum
// chains are latency-bound, and the phases, which both forms compute per
// halo pixel and pair, are a large part of either.
#include <math.h>

#include "bf_fir32.cuh"

namespace bf {
namespace {

constexpr int TW = 32;
constexpr float kQ = 2097152.0f;           // 2^21
constexpr float kInvQ = 1.0f / 2097152.0f;

struct BoxGeo {
    int R, RH, RW, RWp, RBs;
    __host__ __device__ BoxGeo(int R_, int TH)
    {
        R = R_;
        RH = TH + 2 * R;
        RW = TW + 2 * R;
        RWp = (RW + 15) / 16 * 16 + 1;     // odd: lanes on consecutive rows hit distinct banks
        RBs = TW + 1;                      // row-sum buffer stride
    }
    __host__ __device__ size_t bytes() const
    {
        return sizeof(float) * (size_t)RH * RWp            // centred, scaled f
               + sizeof(float2) * (size_t)RH * RWp         // (cos, sin)
               + sizeof(int) * 2 * (size_t)RH * RBs;       // row sums of two planes
    }
};

__device__ __forceinline__ int qz(float v)
{
    return __float2int_rn(fminf(fmaxf(v, -8.f), 8.f) * kQ);
}

template <int TH>
__global__ void __launch_bounds__(4 * TH) k_box32(FwdArgs a)
{
    constexpr int NT = 4 * TH;
    extern __shared__ __align__(16) unsigned char smraw[];
    const BoxGeo G(a.R, TH);
    const int R = a.R;
    float2* cs = reinterpret_cast<float2*>(smraw);                       // RH x RWp
    float* fz = reinterpret_cast<float*>(cs + (size_t)G.RH * G.RWp);      // RH x RWp
    int* rb = reinterpret_cast<int*>(fz + (size_t)G.RH * G.RWp);          // 2 x RH x RBs

    const int by = (blockIdx.y + a.y_tile0) * TH, bx = blockIdx.x * TW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gy0 = by - R, gx0 = bx - R;
    const int set = a.set_tile ? (by / a.set_tile) * a.sets_x + (bx / a.set_tile) : 0;
    const SetHdr hd = a.hdr[set];
    const int cx = tid % TW, cg = tid / TW;        // my column item: column cx, rows 8 cg ..
    const int gx = bx + cx;

    if (hd.F < 0) {          // order above the cap: pass the image through
        for (int i = 0; i < 8; ++i) {
            const int gy = by + cg * 8 + i;
            if (gy < a.H && gx < a.W)
                a.out[(size_t)gy * a.out_pitch + gx] = a.f[(size_t)gy * a.f_pitch + gx];
        }
        return;
    }
    const float c0 = a.c0, inv_c0 = 1.0f / a.c0;
    for (int r = warp; r < G.RH; r += NT / 32) {
        const int gy = gy0 + r;
        const bool rin = gy >= 0 && gy < a.H;
        for (int col = lane; col < G.RW; col += 32) {
            const int x = gx0 + col;
            float v = 0.f;
            if (rin && x >= 0 && x < a.W) v = __ldg(a.f + (size_t)gy * a.f_pitch + x) - c0;
            fz[r * G.RWp + col] = v;
        }
    }
    const float full = full_mass(a.taps, R);
    const float cmass = clipped_mass(a.taps, R, gx, a.W, full);
    float num[8], den[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) num[i] = den[i] = 0.f;
    __syncthreads();

    const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    const int K = hd.F + hd.z;
    const int half = TW / 2;
    for (int k = 0; k < K; ++k) {
        float om_hi = 0.f, om_lo = 0.f, Wk = hd.w0;
        if (k < hd.F) {
            const Pair p = pr[k];
            om_hi = p.om_hi;
            om_lo = p.om_lo;
            Wk = p.W;
        }
        // phases of every in-image halo pixel, 0 elsewhere
        for (int r = warp; r < G.RH; r += NT / 32) {
            const int gy = gy0 + r;
            const bool rin = gy >= 0 && gy < a.H;
            for (int col = lane; col < G.RW; col += 32) {
                const int x = gx0 + col;
                float c = 0.f, sn = 0.f;
                if (rin && x >= 0 && x < a.W) fir32::phase_cs(fz[r * G.RWp + col], om_hi, om_lo, c, sn);
                cs[r * G.RWp + col] = make_float2(c, sn);
            }
        }
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {       // 0: den (c, s), 1: num (f c, f s)
            // rows: item (row, plane, half) -> running sums of 16 outputs
            for (int it = tid; it < G.RH * 4; it += NT) {
                const int r = it % G.RH, q = it / G.RH;
                const int pl = q & 1, hf = q >> 1;
                const float2* row = cs + r * G.RWp + hf * half;
                const float* frow = fz + r * G.RWp + hf * half;
                auto val = [&](int j) {
                    const float2 v = row[j];
                    float w = pl ? v.y : v.x;
                    if (pass) w *= frow[j] * inv_c0;
                    return qz(w);
                };
                unsigned acc = 0;
                for (int j = 0; j <= 2 * R; ++j) acc += (unsigned)val(j);
                int* dst = rb + (size_t)pl * G.RH * G.RBs + r * G.RBs + hf * half;
                dst[0] = (int)acc;
                for (int x = 1; x < half; ++x) {
                    acc += (unsigned)val(x + 2 * R) - (unsigned)val(x - 1);  // exact: fits int32
                    dst[x] = (int)acc;
                }
            }
            __syncthreads();
            // columns of my item (both planes), then demodulate
            {
                const int* c0p = rb + cg * 8 * G.RBs + cx;
                const int* c1p = c0p + (size_t)G.RH * G.RBs;
                long long s0 = 0, s1 = 0;
                for (int j = 0; j <= 2 * R; ++j) {
                    s0 += c0p[j * G.RBs];
                    s1 += c1p[j * G.RBs];
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (i > 0) {
                        s0 += (long long)c0p[(i + 2 * R) * G.RBs] - c0p[(i - 1) * G.RBs];
                        s1 += (long long)c1p[(i + 2 * R) * G.RBs] - c1p[(i - 1) * G.RBs];
                    }
                    const float2 v = cs[(cg * 8 + i + R) * G.RWp + cx + R];
                    const float b0 = (float)s0 * kInvQ, b1 = (float)s1 * kInvQ;
                    if (pass) num[i] = fmaf(Wk, fmaf(v.x, b0, v.y * b1), num[i]);
                    else den[i] = fmaf(Wk, fmaf(v.x, b0, v.y * b1), den[i]);
                }
            }
            __syncthreads();
        }
    }

    if (gx < a.W) {
        const float kap = a.fix_list ? a.fix_kappa : -INFINITY;   // FP32 recheck list
        uint32_t listed = 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gy = by + cg * 8 + i;
            if (gy >= a.H) continue;
            const float rmass = clipped_mass(a.taps, R, gy, a.H, full);
            float v;
            if (den[i] < kap * rmass * cmass) {
                listed |= 1u << i;
                v = a.f[(size_t)gy * a.f_pitch + gx];
            } else if (den[i] > kGuard * rmass * cmass) {
                v = fmaf(__fdiv_rn(num[i], den[i]), c0, c0);
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
                (unsigned)(by + cg * 8 + i) * (unsigned)a.W + (unsigned)gx;
        }
    }
}

template <int TH>
cudaError_t launch_box_t(const FwdArgs& a, cudaStream_t s)
{
    const BoxGeo G(a.R, TH);
    cudaError_t e = cudaFuncSetAttribute(k_box32<TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G.bytes());
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, a.y_tiles > 0 ? a.y_tiles : (a.H + TH - 1) / TH);
    k_box32<TH><<<grid, 4 * TH, G.bytes(), s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Output rows of the running-sum tile for radius R and T-tiles of set_tile
// rows (0: one set), 0 when none fits (the FIR with unit taps serves then).
int box32_rows(int R, int set_tile)
{
    if (R < 1 || R > 63) return 0;
    static const int rows[] = {128, 64, 32};
    for (int th : rows) {
        if (set_tile && set_tile % th) continue;
        if (BoxGeo(R, th).bytes() <= 227 * 1024) return th;
    }
    return 0;
}

cudaError_t launch_box32(const FwdArgs& a, cudaStream_t s)
{
    switch (box32_rows(a.R, a.set_tile)) {
    case 128: return launch_box_t<128>(a, s);
    case 64: return launch_box_t<64>(a, s);
    case 32: return launch_box_t<32>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace bf
