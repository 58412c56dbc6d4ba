// FP32 recheck of the outputs that a 16-bit-plane forward (K3-tc) listed.
//
// At a pixel unlike most of its window the denominator of eq. (f2) is a
// small part of the window's spatial mass, and the terms that cancel down to
// it are of the order of that mass: the 16-bit rounding of the modulated
// planes (and of the vertical pass) is amplified by mass / den.  K3-tc lists
// every output with den < kappa * (g * 1_Omega)(x), per parameter set; this
// kernel recomputes each of them in FP32 by the direct sum of eq. (BF) with
// the set's phi_eps (eq. (approx), the same N, M and folded weights as the
// planes):
//
//   out(x) = f(x) + sum_y g(x - y) phi_eps(d_y) d_y / sum_y g(x - y) phi_eps(d_y),
//   d_y = f(y) - f(x),   phi_eps(d) = w0 [N even] + sum_k W_k cos(omega_k d),
//
// omega_k = omega_0 + k Delta, Delta = 2 / (sqrt(N) sigma_r) (omega_0 = Delta
// for even N, Delta / 2 for odd N).
//
// phi_eps depends on d alone, so one CTA per parameter set first tabulates
// it on a grid s_j = (j - 1) h, j = 0 .. J, of [0, T] (phi_eps is even and
// |d| <= T within a window), then every (output, neighbour) pair reads it by
// 4-point (cubic) Lagrange interpolation, with a first-order correction for
// the exact tail of d.  The interpolation error is at most |phi''''| h^4
// (9/16) / 24 <= 0.0234 (omega_max h)^4 (sum_k W_k <= 1), so h = the
// largest power of two with omega_max h <= 0.054 keeps it under 2e-7; a power
// of two makes every s_j and s / h exact.  A set whose table does not fit the
// launch's shared memory (or a |d| beyond T, possible only for fixed T)
// takes the same value from the sum itself:
//   phi_eps(d) = Re[e^{i omega_0 d} P(z)],  P(z) = sum_k W_k z^k,  z = e^{i Delta d},
// by Horner's rule on the unit circle, with d as an exact head + tail
// (two-sum), Delta d as a head + tail product and one accurate sincosf
// (|Delta d| <= pi whenever |d| <= T).  Table entries come from the same
// routine.  num and den are compensated sums (two-sum per term), then the
// denominator guard and the normalisation of the forward.
//
// One warp per listed pixel (lanes over the (2R+1)^2 window).  A one-CTA
// scan turns the per-set list lengths into offsets, and a persistent grid
// splits all listed pixels evenly (the lists are very uneven: pixels unlike
// their window gather at edges and in noisy tiles); every CTA builds the
// tables of the sets its share touches.  List lengths are read on the
// device, so the launch needs no host synchronisation.
#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr float kTabStep = 0.054f;   // omega_max * h bound of the table grid

// s + c += v, c collecting the rounding error of each addition (two-sum)
__device__ __forceinline__ void comp_add(float& s, float& c, float v)
{
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

struct SetConst {
    float Dhi, Dlo, w0;
    bool odd;
    int K;
};

// phi_eps(dh + dl) from its pair sum (Horner on the unit circle); wk in
// shared memory.
__device__ __forceinline__ float phi_sum(float dh, float dl, const SetConst& c, const float* wk)
{
    const float ph = c.Dhi * dh;
    float pe = fmaf(c.Dhi, dh, -ph);
    pe = fmaf(c.Dhi, dl, pe);
    pe = fmaf(c.Dlo, dh, pe);
    float ang = ph + pe;
    if (c.odd) ang *= 0.5f;
    float s1, c1;
    sincosf(ang, &s1, &c1);
    const float mr = c1, mi = s1;                          // e^{i omega_0 d}
    const float zr = c.odd ? fmaf(c1, c1, -s1 * s1) : c1;
    const float zi = c.odd ? 2.f * c1 * s1 : s1;           // e^{i Delta d}
    float pr_ = 0.f, pi_ = 0.f;
    for (int k = c.K - 1; k >= 0; --k) {
        const float tr = fmaf(-pi_, zi, fmaf(pr_, zr, wk[k]));
        pi_ = fmaf(pr_, zi, pi_ * zr);
        pr_ = tr;
    }
    return fmaf(mr, pr_, -mi * pi_) + c.w0;
}

// Exclusive prefix sum of the per-set list lengths of the launch's sets, in
// one CTA (scan[i] = items before set set0 + i; scan[n_sets] = all items).
__global__ void __launch_bounds__(1024) k_fixup_scan(const unsigned* __restrict__ count, int set0,
                                                     int n_sets, unsigned* __restrict__ scan)
{
    __shared__ unsigned part[1024];
    const int per = (n_sets + 1023) / 1024;
    const int i0 = threadIdx.x * per, i1 = min(n_sets, i0 + per);
    unsigned s = 0;
    for (int i = i0; i < i1; ++i) s += count[set0 + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {        // inclusive scan of the parts
        const unsigned v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int i = i0; i < i1; ++i) {
        scan[i] = run;
        run += count[set0 + i];
    }
    if (threadIdx.x == 1023) scan[n_sets] = part[1023];
}

// Per-set constants and the phi_eps table of `set` (whole CTA).
__device__ void load_set(const FixArgs& a, int set, float* wk, float* tab, SetConst& sc, float& h,
                         float& inv_h, int& J, bool& use_tab)
{
    const SetHdr hd = a.hdr[set];
    const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    __syncthreads();                                   // the previous set's table is done with
    for (int k = threadIdx.x; k < hd.F; k += kThreads) wk[k] = pr[k].W;
    const double scale = sqrt((double)hd.N) * a.sigma_r;
    const double D = 2.0 / scale;
    sc.Dhi = (float)D;
    sc.Dlo = (float)(D - (double)sc.Dhi);
    sc.odd = hd.N & 1;
    sc.w0 = hd.z ? hd.w0 : 0.f;
    sc.K = hd.F;
    // the table grid: omega_max of the set's largest kept pair
    const double om_max = hd.F > 0 ? (sc.odd ? 2.0 * hd.F - 1.0 : 2.0 * hd.F) / scale : 0.0;
    h = inv_h = 0.f;
    J = 0;
    use_tab = false;
    if (om_max > 0.0) {
        const int e = (int)floor(log2((double)kTabStep / om_max));
        h = ldexpf(1.0f, e);
        inv_h = ldexpf(1.0f, -e);
        const double jd = (double)hd.T / (double)h + 4.0;
        if (jd <= (double)a.ntab) {
            J = (int)jd;
            use_tab = true;
        }
    }
    __syncthreads();
    if (use_tab) {
        for (int j = threadIdx.x; j <= J; j += kThreads)
            tab[j] = phi_sum((float)(j - 1) * h, 0.f, sc, wk);
        __syncthreads();
    }
}

// Persistent: CTA b takes items [b T / G, (b + 1) T / G) of the launch's
// T listed outputs in set order (scan gives each set's first item), builds
// the table of every set it meets and hands the items to its warps.
__global__ void __launch_bounds__(kThreads, 4) k_fixup(FixArgs a, const unsigned* __restrict__ scan,
                                                    int n_sets)
{
    extern __shared__ float sm[];
    const int RW = 2 * a.R + 1;
    float* taps = sm;                                  // 2R+1
    float* wk = taps + ((RW + 3) & ~3);                // cap_pairs
    float* tab = wk + ((a.cap_pairs + 3) & ~3);        // phi_eps((j - 1) h), j <= J

    const unsigned total = scan[n_sets];
    const unsigned b0 = (unsigned)(((unsigned long long)blockIdx.x * total) / gridDim.x);
    const unsigned b1 = (unsigned)(((unsigned long long)(blockIdx.x + 1) * total) / gridDim.x);
    if (b0 >= b1) return;                              // whole CTA
    for (int i = threadIdx.x; i < RW; i += kThreads) taps[i] = a.taps[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float full = full_mass(taps, a.R);

    // the set holding item b0: the last i with scan[i] <= b0
    int lo = 0, hi = n_sets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (scan[mid] <= b0) lo = mid;
        else hi = mid - 1;
    }
    for (int si = lo; si < n_sets; ++si) {
        const unsigned s0 = max(scan[si], b0), s1 = min(scan[si + 1], b1);
        if (s0 >= b1) break;
        if (s0 >= s1) continue;                        // (uniform) empty set
        const int set = a.set0 + si;
        SetConst sc;
        float h, inv_h;
        int J;
        bool use_tab;
        load_set(a, set, wk, tab, sc, h, inv_h, J, use_tab);
        const unsigned* list = a.list + (size_t)set * a.fix_cap;
        for (unsigned g = s0 + warp; g < s1; g += kWarps) {
            const unsigned idx = list[g - scan[si]];
            const int gy = (int)(idx / (unsigned)a.W), gx = (int)(idx - (unsigned)gy * a.W);
            const float fx = a.f[(size_t)gy * a.f_pitch + gx];
            float ns = 0.f, nc = 0.f, ds = 0.f, dc = 0.f;
            constexpr int kU = 8;                      // window loads in flight per lane
            // window position of this lane's first neighbour, then advanced by
            // 32 positions per step without a division
            int iy = lane / RW, ix = lane - (lane / RW) * RW;
            for (int p0 = lane; p0 < RW * RW; p0 += 32 * kU) {
                float fv[kU], gv[kU];                  // neighbour value, spatial weight
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int y = gy + iy - a.R, x = gx + ix - a.R;
                    const bool in = p0 + 32 * u < RW * RW && y >= 0 && y < a.H && x >= 0 &&
                                    x < a.W;
                    fv[u] = in ? __ldg(a.f + (size_t)y * a.f_pitch + x)
                               : __int_as_float(0x7fc00000);
                    gv[u] = taps[min(iy, RW - 1)] * taps[min(ix, RW - 1)];
                    ix += 32;
                    while (ix >= RW) {
                        ix -= RW;
                        ++iy;
                    }
                }
                // plain sums over the kU terms of this step, compensated across steps
                float dsum = 0.f, nsum = 0.f;
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    if (isnan(fv[u])) continue;
                    const float fy = fv[u];
                    // d = fy - fx = dh + dl exactly
                    const float dh = fy - fx;
                    const float t = dh - fy;
                    const float dl = (fy - (dh - t)) + (-fx - t);
                    const float q = fabsf(dh) * inv_h;
                    const int j0 = (int)q;
                    float phi;
                    if (use_tab && j0 + 3 <= J) {
                        const float uu = q - (float)j0;
                        const float v0 = tab[j0], v1 = tab[j0 + 1], v2 = tab[j0 + 2],
                                    v3 = tab[j0 + 3];
                        const float um1 = uu - 1.f, um2 = uu - 2.f, up1 = uu + 1.f;
                        const float wa = -uu * um1 * um2 * (1.f / 6.f);
                        const float wb = up1 * um1 * um2 * 0.5f;
                        const float wc = -up1 * uu * um2 * 0.5f;
                        const float wd = up1 * uu * um1 * (1.f / 6.f);
                        phi = fmaf(wa, v0, fmaf(wb, v1, fmaf(wc, v2, wd * v3)));
                        // first-order term of the tail: phi'(s) ~ (v2 - v1) / h
                        phi = fmaf((v2 - v1) * inv_h, dh < 0.f ? -dl : dl, phi);
                    } else {
                        phi = phi_sum(dh, dl, sc, wk);
                    }
                    const float wgt = gv[u] * phi;
                    dsum += wgt;
                    nsum = fmaf(wgt, dh, nsum);
                }
                comp_add(ds, dc, dsum);
                comp_add(ns, nc, nsum);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float ns2 = __shfl_xor_sync(0xffffffffu, ns, off);
                const float nc2 = __shfl_xor_sync(0xffffffffu, nc, off);
                const float ds2 = __shfl_xor_sync(0xffffffffu, ds, off);
                const float dc2 = __shfl_xor_sync(0xffffffffu, dc, off);
                comp_add(ns, nc, ns2);
                nc += nc2;
                comp_add(ds, dc, ds2);
                dc += dc2;
            }
            if (lane == 0) {
                const float num = ns + nc, den = ds + dc;
                const float rmass = clipped_mass(taps, a.R, gy, a.H, full);
                const float cmass = clipped_mass(taps, a.R, gx, a.W, full);
                float v;
                if (den > kGuard * rmass * cmass) {
                    v = fx + __fdiv_rn(num, den);
                } else {
                    v = fx;
                    atomicAdd(a.n_guarded, 1ull);
                }
                a.out[(size_t)gy * a.out_pitch + gx] = v;
            }
        }
    }
}

}  // namespace

size_t fixup_smem_bytes(int R, int cap_pairs, int ntab)
{
    const size_t RW = 2 * (size_t)R + 1;
    return sizeof(float) * (((RW + 3) & ~(size_t)3) + (((size_t)cap_pairs + 3) & ~(size_t)3) +
                            (size_t)ntab + 1);
}

// Table entries for a plan: enough for every set whose N fits n_cap (T <=
// pi sigma_r sqrt(N) / 2 and omega_max <= sqrt(N) / sigma_r, with the step
// at least 0.027 / omega_max, give J <= (pi / 2) N / 0.027 + 4 < 59 N + 4),
// but at most kMaxTab entries; sets with a
// longer table take the direct sums.  48 KB: four CTAs (32 warps) per SM.
int fixup_table_entries(int n_cap)
{
    constexpr long long kMaxTab = 12288;
    long long want = 59ll * n_cap + 8;
    return (int)(want < kMaxTab ? want : kMaxTab);
}

cudaError_t launch_fixup(const FixArgs& a, int n_sets, cudaStream_t s)
{
    const size_t smem = fixup_smem_bytes(a.R, a.cap_pairs, a.ntab);
    if (smem > 227 * 1024 || n_sets < 1 || !a.scan) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fixup, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_fixup_scan<<<1, 1024, 0, s>>>(a.count, a.set0, n_sets, a.scan);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fixup<<<a.n_ctas, kThreads, smem, s>>>(a, a.scan, n_sets);
    return cudaGetLastError();
}

}  // namespace bf
