// SHIFTABLE-BF with the raised-polynomial range kernel (Sec. 1.3, eqs. (RP),
// (RPconv)): phi(s) = (1 - s^2 / (2 N sigma_r^2))^N, N = max(1, ceil(T^2 /
// (2 sigma_r^2))), the positivity / monotonicity threshold of Sec. 1.3.
//
// The kernel is shiftable because phi(f(y) - f(x)) is a polynomial of degree
// 2N in f(y) whose coefficients depend on f(x) (eqs. (f1), (f2) with a
// polynomial basis).  The monomial basis f^k the paper names cancels
// catastrophically in FP32 (coefficients of size ~2^N summing to O(1)), so
// the GB300 form takes another basis of the same polynomial space: with
// u = (f - c) / h mapping the values of a parameter set's region onto
// [-1, 1], the Lagrange polynomials L_i(u) of the n = 2N + 1 Chebyshev
// points v_i = cos((2i + 1) pi / (2n)).  For every u_x,
//
//   K(u_y, u_x) = (1 - beta (u_y - u_x)^2)^N = sum_i K(v_i, u_x) L_i(u_y),
//   beta = h^2 / (2 N sigma_r^2),
//
// exactly (interpolation of a degree-2N polynomial at 2N + 1 points), so the
// planes are G_i = L_i(u), F_i = u L_i(u) and the coefficients of eqs. (f1),
// (f2) are c_i(u_x) = K(v_i, u_x), which lie in [0, 1]; sum_i |L_i(u)| is
// the Lebesgue constant of Chebyshev points (about (2/pi) log n + 1), so no
// term is much larger than the result.  L_i comes from the barycentric
// formula L_i(u) = (l_i / (u - v_i)) / sum_k (l_k / (u - v_k)), l_k =
// (-1)^k sin((2k + 1) pi / (2n)), stable for these points.
//
// T is the range of f over each set's region (the T-tile grown by R, or the
// image): every pair of values the expansion of a region represents is then
// within [-T, T], so 1 - beta (u_y - u_x)^2 >= 0 on all of [-1, 1]^2 and the
// expansion stays bounded.  With Algorithm 1's T (the largest difference
// within one window) the polynomial would be evaluated, through the basis,
// at value pairs up to the region's range apart, where it grows like
// (range^2 / T^2)^N.
//
// Kernels: k_poly_range (max and min of f per set region), k_poly_params
// (N, c, h, beta and the n nodes / weights per set, FP64), k_poly32 (fused
// tile: per two terms, modulate, the FP32 FIR of the other forward kernels,
// demodulate; out = c + h num / den with the denominator guard).
#include <math.h>

#include "bf_fir32.cuh"

namespace bf {
namespace {

using fir32::Geo;

constexpr double kPi = 3.14159265358979323846;

// float -> unsigned with the same order (so that atomicMax / atomicMin on
// the codes order the floats)
__device__ __forceinline__ unsigned ord_enc(float v)
{
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

constexpr int kRangeThreads = 256;

// max and min of f over set regions: mm[2 s] = code of the max of f,
// mm[2 s + 1] = code of the max of -f (both cleared to 0, below every code).
// With T-tiles, block b takes set b's region (the T-tile grown by R,
// clipped); with one set, the blocks stride over the image.
__global__ void __launch_bounds__(kRangeThreads)
k_poly_range(const float* __restrict__ f, size_t pitch, int H, int W, int R, int set_tile,
             int sets_x, unsigned* __restrict__ mm)
{
    float mx = -INFINITY, nmn = -INFINITY;     // max of f, max of -f
    int set = 0;
    if (set_tile) {
        set = blockIdx.x;
        const int ty = set / sets_x, tx = set - ty * sets_x;
        const int y0 = max(0, ty * set_tile - R), y1 = min(H, (ty + 1) * set_tile + R);
        const int x0 = max(0, tx * set_tile - R), x1 = min(W, (tx + 1) * set_tile + R);
        const int w = x1 - x0;
        for (int i = threadIdx.x; i < (y1 - y0) * w; i += kRangeThreads) {
            const int y = y0 + i / w, x = x0 + i % w;
            const float v = __ldg(f + (size_t)y * pitch + x);
            mx = fmaxf(mx, v);
            nmn = fmaxf(nmn, -v);
        }
    } else {
        const size_t n = (size_t)H * W;
        for (size_t i = (size_t)blockIdx.x * kRangeThreads + threadIdx.x; i < n;
             i += (size_t)gridDim.x * kRangeThreads) {
            const float v = __ldg(f + (i / W) * pitch + i % W);
            mx = fmaxf(mx, v);
            nmn = fmaxf(nmn, -v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        nmn = fmaxf(nmn, __shfl_xor_sync(0xffffffffu, nmn, o));
    }
    if ((threadIdx.x & 31) == 0 && mx > -INFINITY) {
        atomicMax(mm + 2 * set, ord_enc(mx));
        atomicMax(mm + 2 * set + 1, ord_enc(nmn));
    }
}

// One block per set: N, centre c, half-range h, beta and the Chebyshev nodes
// v_k with their barycentric weights (FP64, rounded to FP32 once).
// Header fields: N, M = 0, F = n = 2N + 1 (terms), z = 0, w0 = beta, T,
// pad0 = c, pad1 = h.  Node k: om_hi = v_k, om_lo = l_k.
__global__ void __launch_bounds__(128) k_poly_params(PolyParamsArgs a)
{
    const int set = blockIdx.x;
    double T, c, h;
    if (a.mm) {
        const double mx = (double)ord_dec(a.mm[2 * set]);
        const double mn = -(double)ord_dec(a.mm[2 * set + 1]);
        T = mx - mn;
        c = 0.5 * (mx + mn);
        h = 0.5 * T;
    } else {
        T = a.t_fixed;
        c = 0.5 * a.value_range;
        h = 0.5 * a.value_range;
    }
    if (!(h > 0.0)) h = 1.0;     // a flat region: any scale (every u is 0)
    const double n0 = (T * T) / (2.0 * a.sigma_r * a.sigma_r);
    const double cn = ceil(n0);
    const int N = cn < 1.0 ? 1 : (cn > 1e9 ? 1000000000 : (int)cn);
    SetHdr hd;
    hd.M = 0;
    hd.z = 0;
    hd.T = (float)T;
    hd.pad0 = (float)c;
    hd.pad1 = (float)h;
    hd.N = N;
    if (N > a.n_cap) {
        if (threadIdx.x == 0) {
            hd.F = -1;
            hd.w0 = 0.f;
            a.hdr[set] = hd;
            atomicOr(a.status, kDevOrder);
        }
        return;
    }
    const int n = 2 * N + 1;
    Pair* nd = a.nodes + (size_t)set * a.cap_nodes;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double t = (2.0 * k + 1.0) * kPi / (2.0 * n);
        Pair p;
        p.om_hi = (float)cos(t);
        p.om_lo = (float)((k & 1) ? -sin(t) : sin(t));
        p.W = 0.f;
        p.pad = 0.f;
        nd[k] = p;
    }
    if (threadIdx.x == 0) {
        hd.F = n;
        hd.w0 = (float)(h * h / (2.0 * (double)N * a.sigma_r * a.sigma_r));
        a.hdr[set] = hd;
    }
}

// K(v, u) = (1 - beta (v - u)^2)^N, 0 where the base is not positive
__device__ __forceinline__ float poly_coef(float v, float u, float beta, float N)
{
    const float d = v - u;
    const float q = beta * d * d;
    return q < 1.f ? expf(N * log1pf(-q)) : 0.f;
}

template <int TH, int TW>
__global__ void __launch_bounds__(TH * TW / 8) k_poly32(FwdArgs a)
{
    constexpr int NT = TH * TW / 8;
    constexpr int NW = NT / 32;
    extern __shared__ float sm[];
    const Geo G(a.R, TH, TW);
    const int R = a.R;
    const size_t reg = (size_t)G.RH * G.RWp;
    float* usm = sm;                       // u = (f - c) / h, 0 outside the image
    float* asm_ = usm + reg;               // L_a(u)
    float* bsm = asm_ + reg;               // L_b(u)
    float* ism = bsm + reg;                // 1 / sum_k l_k / (u - v_k), 0 outside the image
    float* hsm = ism + reg;                // 4 x RHp x TW row-filtered planes
    float* gz = hsm + 4 * (size_t)G.RHp * TW;
    float2* nod = reinterpret_cast<float2*>(gz + G.ngz + (G.ngz & 1));   // (v_k, l_k)
    const size_t hplane = (size_t)G.RHp * TW;

    const int by = blockIdx.y * TH, bx = blockIdx.x * TW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gy0 = by - R, gx0 = bx - R;
    const int set = a.set_tile ? (by / a.set_tile) * a.sets_x + (bx / a.set_tile) : 0;
    const SetHdr hd = a.hdr[set];
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
    const int n = hd.F;
    const float beta = hd.w0, c = hd.pad0, h = hd.pad1, Nf = (float)hd.N;
    const float inv_h = 1.0f / h;
    const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    for (int k = tid; k < n; k += NT) nod[k] = make_float2(pr[k].om_hi, pr[k].om_lo);
    for (int i = tid; i < G.ngz; i += NT) {
        const int t = i - 8;
        gz[i] = (t >= 0 && t <= 2 * R) ? a.taps[t] : 0.f;
    }
    for (int i = tid; i < (G.RHp - G.RH) * TW; i += NT)
        for (int q = 0; q < 4; ++q) hsm[q * hplane + (size_t)G.RH * TW + i] = 0.f;
    __syncthreads();
    // scaled values and barycentric denominators of the block + halo
    for (int r = warp; r < G.RH; r += NW) {
        const int gy = gy0 + r;
        const bool rin = gy >= 0 && gy < a.H;
        for (int col = lane; col < G.RWp; col += 32) {
            const int x = gx0 + col;
            float u = 0.f, is = 0.f;
            if (rin && col < G.RW && x >= 0 && x < a.W) {
                u = (__ldg(a.f + (size_t)gy * a.f_pitch + x) - c) * inv_h;
                float S = 0.f;
                for (int k = 0; k < n; ++k) {
                    float d = u - nod[k].x;
                    d = d == 0.f ? 1e-30f : d;
                    S += __fdividef(nod[k].y, d);
                }
                is = 1.0f / S;
            }
            usm[r * G.RWp + col] = u;
            ism[r * G.RWp + col] = is;
        }
    }
    const float full = full_mass(a.taps, R);
    const float cmass = clipped_mass(a.taps, R, gx, a.W, full);
    float num[8], den[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) num[i] = den[i] = 0.f;
    __syncthreads();

    for (int ta = 0; ta < n; ta += 2) {
        const int tb = ta + 1;
        const float2 na = nod[ta];
        const float2 nb = tb < n ? nod[tb] : make_float2(0.f, 0.f);
        // (1) modulate: L_a, L_b at every halo pixel (0 outside the image)
        for (int r = warp; r < G.RH; r += NW) {
            for (int col = lane; col < G.RWp; col += 32) {
                const int e = r * G.RWp + col;
                const float u = usm[e], is = ism[e];
                float da = u - na.x, db = u - nb.x;
                da = da == 0.f ? 1e-30f : da;
                db = db == 0.f ? 1e-30f : db;
                asm_[e] = __fdividef(na.y, da) * is;
                bsm[e] = tb < n ? __fdividef(nb.y, db) * is : 0.f;
            }
        }
        __syncthreads();
        // (2) rows: planes (u L_a, u L_b, L_a, L_b)
        fir32::row_pass<TW, true>(G, usm, nullptr, asm_, bsm, gz, hsm, tid, NT);
        __syncthreads();
        // (3) columns of my item, then demodulate with c_a(u_x), c_b(u_x)
        {
            float acc[4][8];
            fir32::col_pass<TW>(G, hsm, gz, o, rb, acc);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float ux = usm[(rb * 8 + i + R) * G.RWp + o + R];
                const float ca = poly_coef(na.x, ux, beta, Nf);
                const float cb = tb < n ? poly_coef(nb.x, ux, beta, Nf) : 0.f;
                num[i] = fmaf(ca, acc[0][i], fmaf(cb, acc[1][i], num[i]));
                den[i] = fmaf(ca, acc[2][i], fmaf(cb, acc[3][i], den[i]));
            }
        }
        __syncthreads();
    }

    if (gx < a.W) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gy = by + rb * 8 + i;
            if (gy >= a.H) continue;
            const float rmass = clipped_mass(a.taps, R, gy, a.H, full);
            float v;
            if (den[i] > kGuard * rmass * cmass) {
                v = fmaf(h, __fdiv_rn(num[i], den[i]), c);
            } else {
                v = a.f[(size_t)gy * a.f_pitch + gx];
                atomicAdd(a.n_guarded, 1ull);
            }
            a.out[(size_t)gy * a.out_pitch + gx] = v;
        }
    }
}

size_t poly_smem_bytes(int R, int th, int tw, int cap_nodes)
{
    const Geo G(R, th, tw);
    return sizeof(float) * (G.floats(tw, 4) + (G.ngz & 1) + 2 * (size_t)cap_nodes);
}

template <int TH, int TW>
cudaError_t launch_poly_tile(const FwdArgs& a, cudaStream_t s)
{
    const size_t smem = poly_smem_bytes(a.R, TH, TW, a.cap_pairs);
    cudaError_t e = cudaFuncSetAttribute(k_poly32<TH, TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    k_poly32<TH, TW><<<grid, TH * TW / 8, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

void poly_tile(int R, int cap_nodes, int* th, int* tw)
{
    static const int shapes[][2] = {{64, 32}, {32, 32}, {16, 16}};
    for (auto& sh : shapes)
        if (poly_smem_bytes(R, sh[0], sh[1], cap_nodes) <= 227 * 1024) {
            *th = sh[0];
            *tw = sh[1];
            return;
        }
    *th = *tw = 0;
}

cudaError_t launch_poly_range(const float* f, size_t pitch, int H, int W, int R, int set_tile,
                              int sets_x, int n_sets, unsigned* mm, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(mm, 0, sizeof(unsigned) * 2 * n_sets, s);
    if (e != cudaSuccess) return e;
    const int blocks = set_tile ? n_sets : 2 * 152;
    k_poly_range<<<blocks, kRangeThreads, 0, s>>>(f, pitch, H, W, R, set_tile, sets_x, mm);
    return cudaGetLastError();
}

cudaError_t launch_poly_params(const PolyParamsArgs& a, cudaStream_t s)
{
    k_poly_params<<<a.n_sets, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_poly32(const FwdArgs& a, cudaStream_t s)
{
    int th = 0, tw = 0;
    poly_tile(a.R, a.cap_pairs, &th, &tw);
    if (th == 64 && tw == 32) return launch_poly_tile<64, 32>(a, s);
    if (th == 32 && tw == 32) return launch_poly_tile<32, 32>(a, s);
    if (th == 16 && tw == 16) return launch_poly_tile<16, 16>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace bf
