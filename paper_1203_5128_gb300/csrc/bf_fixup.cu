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
// phi_eps depends on d alone, so every CTA first tabulates it for the sets
// its share of the list touches: nodes s_j = j h of [0, T] (phi_eps is even
// and |d| <= T within a window), each interval [s_j, s_j+1] holding the
// coefficients of the cubic Hermite interpolant of phi_eps (values and
// slopes at both ends) in u = |d| / h - j.  A pair (output, neighbour)
// reads the float4 of the interval around |d| and evaluates the cubic at u,
// the exact tail of d folded into u.  The interpolant's error is at most
// h^4 max|phi_eps''''| / 384 <= h^4 S4 / 384, S4 = sum_k W_k omega_k^4 (the
// kernel's fourth spectral moment, about 3 / sigma_r^4 for the binomial
// weights, far below omega_max^4), so h = the largest power of two with
// h^4 S4 <= 384e-8 keeps it under 1e-8; a power of two makes every s_j and
// |d| / h exact, and the interval index comes from the bits of a float (no
// conversion instructions).  A set whose table does not fit the launch's
// shared memory takes phi_eps from the sum itself, and so does an output
// with a |d| beyond T (possible only for fixed T), which is redone:
//   phi_eps(d) = Re[e^{i omega_0 d} P(z)],  P(z) = sum_k W_k z^k,  z = e^{i Delta d},
// by Horner's rule on the unit circle, with d as an exact head + tail
// (two-sum), Delta d as a head + tail product and one accurate sincosf
// (|Delta d| <= pi whenever |d| <= T).  The nodes come from the same
// routine, phi_eps' from the same Horner pass with the weights W_k omega_k.
// num and den are compensated sums, then the denominator guard and the
// normalisation of the forward.
//
// One warp per listed pixel (lanes over the (2R+1)^2 window).  The window's
// positions are a per-CTA table of (g(dy) g(dx), pointer offset dy pitch +
// dx) as two arrays, padded with zero weights to whole steps of the
// lanes' loads (steps of 16 loads per lane, the last one of 8 where that
// pads less; the offsets are read to issue the loads, the weights when the
// terms are summed, so that no weight waits in a register): an
// output whose window lies inside the image reads its neighbours through it
// with no bounds test; an output near the border walks the window with the
// bounds tests.  A one-CTA scan turns the per-set list lengths into
// offsets, and a persistent grid splits all listed pixels evenly (the lists
// are very uneven: pixels unlike their window gather at edges and in noisy
// tiles).  List lengths are read on the device, so the launch needs no host
// synchronisation.
#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kU = 16;               // window loads in flight per lane (inside the image)
constexpr int kUB = 8;               // the same near the border, and in a last half step
constexpr int kPad = 32 * kUB;       // the window table's length is a multiple of this

template <int N>
struct Int {
    static constexpr int value = N;
};
constexpr float kTabTol4 = 3.84e-6f; // 384 * 1e-8: h^4 S4 bound of the node grid

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
// shared memory.  Out of line: only sets whose nodes do not fit take it.
__device__ __noinline__ float phi_sum(float dh, float dl, const SetConst& c, const float* wk)
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

// phi_eps(d) and phi_eps'(d) for a d exact in FP32 (the node grid): the
// same Horner pass with the weights W_k and W_k omega_k
__device__ __forceinline__ void phi_node(float d, const SetConst& c, const float* wk,
                                         const float* wkw, float& phi, float& dphi)
{
    const float ph = c.Dhi * d;
    float pe = fmaf(c.Dhi, d, -ph);
    pe = fmaf(c.Dlo, d, pe);
    float ang = ph + pe;
    if (c.odd) ang *= 0.5f;
    float s1, c1;
    sincosf(ang, &s1, &c1);
    const float mr = c1, mi = s1;
    const float zr = c.odd ? fmaf(c1, c1, -s1 * s1) : c1;
    const float zi = c.odd ? 2.f * c1 * s1 : s1;
    float pr_ = 0.f, pi_ = 0.f, qr = 0.f, qi = 0.f;
    for (int k = c.K - 1; k >= 0; --k) {
        const float tr = fmaf(-pi_, zi, fmaf(pr_, zr, wk[k]));
        pi_ = fmaf(pr_, zi, pi_ * zr);
        pr_ = tr;
        const float ur = fmaf(-qi, zi, fmaf(qr, zr, wkw[k]));
        qi = fmaf(qr, zi, qi * zr);
        qr = ur;
    }
    phi = fmaf(mr, pr_, -mi * pi_) + c.w0;
    dphi = -fmaf(mr, qi, mi * qr);                     // -Im[e^{i omega_0 d} Q(z)]
}

// The interpolation table of one set, read by every pair of its outputs.
struct Tab {
    const float4* c;        // interval j: (phi_eps(s_j), h phi_eps'(s_j), c2_j, c3_j)
    float inv_h;
    unsigned J;             // intervals, j = 0 .. J - 1 (0: no table)
};

// phi_eps(dh + dl), |dl| <= ulp(dh) / 2: the cubic of the interval around
// |dh| at u = |dh| / h - j (exact) plus the tail dl / h (its rounding in u
// moves phi_eps by at most h max|phi_eps'| 2^-24 < 3e-9).  kGeneral takes
// the pair sum where the table does not reach (or there is none); else the
// index is clamped to the table and jmax records it, so that the caller
// can redo an output where some lane left the table.
template <bool kGeneral>
__device__ __forceinline__ float phi_at(float dh, float dl, const Tab& t, const SetConst& sc,
                                        const float* wk, unsigned& jmax)
{
    // j = round(|dh| / h - 1/2) by the bits of 1.5 2^23 + (|dh| / h - 1/2), where
    // the FP32 spacing is 1: floor(|dh| / h), or one less when |dh| / h is a
    // whole number (then u = 1 and the cubic gives the next node exactly)
    const float ad = fabsf(dh);
    const float tq = fmaf(ad, t.inv_h, -0.5f) + 12582912.0f;
    unsigned j = (unsigned)(__float_as_int(tq) - 0x4B400000);
    if (kGeneral) {
        if (j >= t.J) return phi_sum(dh, dl, sc, wk);
    } else {
        jmax = max(jmax, j);
        j = min(j, t.J - 1u);
    }
    const float4 c = t.c[j];
    // |d| = |dh| + sign(dh) dl
    const float sdl = __int_as_float(__float_as_int(dl) ^ (__float_as_int(dh) & (int)0x80000000));
    const float u = fmaf(sdl, t.inv_h, fmaf(ad, t.inv_h, 12582912.0f - tq));
    return fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
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

// Per-set constants and the interpolation table of `set` (whole CTA);
// n_tab float4 entries fit.
__device__ void load_set(const FixArgs& a, int set, float* wk, float* wkw, float4* tab,
                         int n_tab, SetConst& sc, Tab& t)
{
    const SetHdr hd = a.hdr[set];
    const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    __syncthreads();                                   // the previous set's table is done with
    for (int k = threadIdx.x; k < hd.F; k += kThreads) {
        const Pair q = pr[k];
        wk[k] = q.W;
        wkw[k] = q.W * q.om_hi;
    }
    // S4 = sum_k W_k omega_k^4, by every warp alike (the butterfly leaves the
    // same sum in every lane)
    float s4 = 0.f;
    for (int k = threadIdx.x & 31; k < hd.F; k += 32) {
        const Pair q = pr[k];
        const float o2 = q.om_hi * q.om_hi;
        s4 = fmaf(q.W * o2, o2, s4);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s4 += __shfl_xor_sync(0xffffffffu, s4, off);
    // Delta = 2 / (sqrt(N) sigma_r) as FP32 head + tail: the first pair's
    // frequency is Delta (even N) or Delta / 2 (odd N), stored the same way
    // (all in FP32: these are per-set constants every thread forms)
    sc.odd = hd.N & 1;
    sc.w0 = hd.z ? hd.w0 : 0.f;
    sc.K = hd.F;
    t.c = tab;
    t.inv_h = 0.f;
    t.J = 0;
    sc.Dhi = sc.Dlo = 0.f;
    float h = 0.f;
    if (hd.F > 0) {
        const Pair first = pr[0];
        const float two = sc.odd ? 2.f : 1.f;
        sc.Dhi = first.om_hi * two;
        sc.Dlo = first.om_lo * two;
        // h = the largest power of two with h^4 S4 <= 384e-8
        const float x = sqrtf(sqrtf(kTabTol4 / s4));
        const int e = ((__float_as_int(x) >> 23) & 255) - 127;          // floor(log2 x)
        if (s4 > 0.f && e > -120 && e < 120) {
            const float inv_h = __int_as_float((127 - e) << 23);
            const float jd = ceilf(hd.T * inv_h) + 1.f;   // intervals 0 .. J - 1 cover [0, T + h]
            if (jd < (float)n_tab) {                     // entries 0 .. J
                h = __int_as_float((e + 127) << 23);
                t.inv_h = inv_h;
                t.J = (unsigned)jd;
            }
        }
    }
    __syncthreads();
    if (t.J) {
        // nodes: (phi_eps(s_j), h phi_eps'(s_j)) in the first half of entry j
        float2* e2 = reinterpret_cast<float2*>(tab);
        for (int j = threadIdx.x; j <= (int)t.J; j += kThreads) {
            float v, dv;
            phi_node((float)j * h, sc, wk, wkw, v, dv);
            e2[2 * j] = make_float2(v, dv * h);
        }
        __syncthreads();
        // the cubic of interval j, v(u) = p0 + u (m0 + u (c2 + u c3)), in the second half
        for (int j = threadIdx.x; j < (int)t.J; j += kThreads) {
            const float2 n0 = e2[2 * j], n1 = e2[2 * j + 2];
            const float dp = n1.x - n0.x;
            e2[2 * j + 1] = make_float2(fmaf(3.f, dp, -fmaf(2.f, n0.y, n1.y)),
                                        fmaf(-2.f, dp, n0.y + n1.y));
        }
        __syncthreads();
    }
}

// The partial sums (per lane, compensated across steps) of num and den of
// one output over its window.
template <bool kGeneral>
__device__ __forceinline__ void window_sums(const FixArgs& a, const int* woff, const float* wwt,
                                            int RW2p, const float* taps, const Tab& t,
                                            const SetConst& sc, const float* wk, int gy, int gx,
                                            float fx, bool inside, float& ns, float& nc,
                                            float& ds, float& dc, unsigned& jmax)
{
    const int lane = threadIdx.x & 31, RW = 2 * a.R + 1, RW2 = RW * RW;
    ns = nc = ds = dc = 0.f;
    // one neighbour: d = fy - fx = dh + dl exactly, its weight g phi_eps(d)
    auto pair = [&](float fy, float gw, float& dsum, float& nsum) {
        const float dh = fy - fx;
        const float tt = dh - fy;
        const float dl = (fy - (dh - tt)) + (-fx - tt);
        const float wgt = gw * phi_at<kGeneral>(dh, dl, t, sc, wk, jmax);
        dsum += wgt;
        nsum = fmaf(wgt, dh, nsum);
    };
    if (inside) {
        // the window lies in the image: positions from the table, no tests
        const float* fc = a.f + (size_t)gy * a.f_pitch + gx;
        // one step of kN positions per lane: plain sums over its terms,
        // compensated across steps
        auto step = [&](int p0, auto n_tag) {
            constexpr int kN = decltype(n_tag)::value;
            float fv[kN];
#pragma unroll
            for (int u = 0; u < kN; ++u) fv[u] = __ldg(fc + woff[p0 + 32 * u]);
            float dsum = 0.f, nsum = 0.f;
#pragma unroll
            for (int u = 0; u < kN; ++u) pair(fv[u], wwt[p0 + 32 * u], dsum, nsum);
            comp_add(ds, dc, dsum);
            comp_add(ns, nc, nsum);
        };
        int p0 = lane;
        for (; p0 + 32 * (kU - 1) < RW2p; p0 += 32 * kU) step(p0, Int<kU>{});
        if (p0 < RW2p) step(p0, Int<kUB>{});          // RW2p a multiple of 32 kUB
    } else {
        // near the border: walk the window, neighbours outside the image skipped
        int iy = lane / RW, ix = lane - (lane / RW) * RW;
        for (int p0 = lane; p0 < RW2; p0 += 32 * kUB) {
            float fv[kUB], gv[kUB];
#pragma unroll
            for (int u = 0; u < kUB; ++u) {
                const int y = gy + iy - a.R, x = gx + ix - a.R;
                const bool in = p0 + 32 * u < RW2 && y >= 0 && y < a.H && x >= 0 && x < a.W;
                fv[u] = in ? __ldg(a.f + (size_t)y * a.f_pitch + x) : fx;
                gv[u] = in ? taps[min(iy, RW - 1)] * taps[min(ix, RW - 1)] : 0.f;
                ix += 32;
                while (ix >= RW) {
                    ix -= RW;
                    ++iy;
                }
            }
            float dsum = 0.f, nsum = 0.f;
#pragma unroll
            for (int u = 0; u < kUB; ++u) pair(fv[u], gv[u], dsum, nsum);
            comp_add(ds, dc, dsum);
            comp_add(ns, nc, nsum);
        }
    }
}

// Persistent: CTA b takes items [b T / G, (b + 1) T / G) of the launch's
// T listed outputs in set order (scan gives each set's first item), builds
// the table of every set it meets and hands the items to its warps.
__global__ void __launch_bounds__(kThreads, 3) k_fixup(FixArgs a, const unsigned* __restrict__ scan,
                                                    int n_sets)
{
    extern __shared__ float4 sm4[];
    const int RW = 2 * a.R + 1, RW2 = RW * RW;
    const int RW2p = (RW2 + kPad - 1) / kPad * kPad;
    float4* tab = sm4;                                             // ntab / 4
    int* woff = reinterpret_cast<int*>(tab + a.ntab / 4);          // RW2p
    float* wwt = reinterpret_cast<float*>(woff + RW2p);            // RW2p
    float* taps = wwt + RW2p;                                      // 2R+1
    float* wk = taps + ((RW + 3) & ~3);                            // cap_pairs
    float* wkw = wk + ((a.cap_pairs + 3) & ~3);                    // cap_pairs

    const unsigned total = scan[n_sets];
    const unsigned b0 = (unsigned)(((unsigned long long)blockIdx.x * total) / gridDim.x);
    const unsigned b1 = (unsigned)(((unsigned long long)(blockIdx.x + 1) * total) / gridDim.x);
    if (b0 >= b1) return;                              // whole CTA
    for (int i = threadIdx.x; i < RW; i += kThreads) taps[i] = a.taps[i];
    __syncthreads();
    // window positions: spatial weight and pointer offset from the centre
    // (zero weight, offset 0 in the padding)
    for (int p = threadIdx.x; p < RW2p; p += kThreads) {
        const int iy = p / RW, ix = p - iy * RW;
        const int off = (iy - a.R) * (int)a.f_pitch + (ix - a.R);
        woff[p] = p < RW2 ? off : 0;
        wwt[p] = p < RW2 ? taps[iy] * taps[ix] : 0.f;
    }
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
        Tab t;
        load_set(a, set, wk, wkw, tab, a.ntab / 4, sc, t);   // (its first barrier covers the window table)
        const unsigned* list = a.list + (size_t)set * a.fix_cap;
        for (unsigned g = s0 + warp; g < s1; g += kWarps) {
            const unsigned idx = list[g - scan[si]];
            const int gy = (int)(idx / (unsigned)a.W), gx = (int)(idx - (unsigned)gy * a.W);
            const float fx = a.f[(size_t)gy * a.f_pitch + gx];
            const bool inside = gy >= a.R && gy + a.R < a.H && gx >= a.R && gx + a.R < a.W;
            float ns, nc, ds, dc;
            unsigned jmax = 0;
            bool general = t.J == 0;                   // (uniform)
            if (!general) {
                window_sums<false>(a, woff, wwt, RW2p, taps, t, sc, wk, gy, gx, fx, inside, ns, nc, ds,
                                   dc, jmax);
                general = __any_sync(0xffffffffu, jmax >= t.J);
            }
            if (general)                               // a |d| beyond the table: the pair sums
                window_sums<true>(a, woff, wwt, RW2p, taps, t, sc, wk, gy, gx, fx, inside, ns, nc, ds,
                                  dc, jmax);
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
    const size_t RW = 2 * (size_t)R + 1, step = kPad;
    const size_t RW2p = (RW * RW + step - 1) / step * step;
    return sizeof(float) * ((size_t)ntab + 2 * RW2p + ((RW + 3) & ~(size_t)3) +
                            2 * (((size_t)cap_pairs + 3) & ~(size_t)3));
}

// Table floats for a plan (four per entry): enough for every set whose N
// fits n_cap (T <= pi sigma_r sqrt(N) / 2, S4 < 3 / sigma_r^4 and h above
// half its bound give J + 1 < 93.4 sqrt(N) + 3 entries), but at most
// kMaxTab floats; sets with more take the pair sums.  With the window table
// (20 KB at R = 24) three CTAs (24 warps) fit an SM.
int fixup_table_entries(int n_cap)
{
    constexpr long long kMaxTab = 12288;
    const long long want = 4 * ((long long)(93.5 * sqrt((double)n_cap)) + 4);
    return (int)(want < kMaxTab ? want : kMaxTab);
}

cudaError_t launch_fixup(const FixArgs& a, int n_sets, cudaStream_t s)
{
    const size_t smem = fixup_smem_bytes(a.R, a.cap_pairs, a.ntab);
    if (smem > 227 * 1024 || n_sets < 1 || !a.scan || a.R > 63) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fixup, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    // the grid splits the listed outputs evenly; every CTA builds the node
    // grids of the sets it meets, so a launch over few sets (a band of the
    // host path) takes one CTA per set, never fewer than one per SM (an
    // image-wide T is one set with all of the image's listed outputs), and
    // at most the CTAs that fit at once
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fixup, kThreads, smem);
    if (e != cudaSuccess) return e;
    const int n_ctas = max(1, min(sms * max(per, 1), max(n_sets, sms)));
    k_fixup_scan<<<1, 1024, 0, s>>>(a.count, a.set0, n_sets, a.scan);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fixup<<<n_ctas, kThreads, smem, s>>>(a, a.scan, n_sets);
    return cudaGetLastError();
}

}  // namespace bf
