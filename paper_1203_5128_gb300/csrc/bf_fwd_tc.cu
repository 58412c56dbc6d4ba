// K3-tc: fused SHIFTABLE-BF forward with FP16 / BF16 planes on the 5th-gen
// tensor cores (tcgen05, accumulators in TMEM).
//
// Same method as K3 (Sec. 1.2, eqs. (f1)-(f2) with phi_eps of eq. (approx)):
// per kept pair, modulate, Gaussian-filter the four planes, demodulate and
// accumulate num / den.  The difference is step 3, the spatial Gaussian: the
// separable FIR over a tile is written as two dense products with constant
// banded Toeplitz matrices, which is exactly the shape tcgen05.mma executes:
//
//   vertical   D1[y, (p, j)] = sum_r Gv[y, r] * P[(p, j), r]      M = 128 rows y
//   horizontal D2[y, (p, x)] = sum_j V_p[y, j] * Gh[x, j]          (per plane p)
//
// with Gv[y, r] = g(r - y - R), Gh[x, j] = g(j - x - R) (zero off the band),
// P the four modulated planes of the tile + halo stored K-major (r fastest),
// and V_p = D1 converted to FP16/BF16 by the threads (TMEM -> registers ->
// shared memory, K-major with j fastest, so no transpose is needed).  All
// operands are K-major, no swizzle; accumulation is FP32 in TMEM.  Phases
// and the demodulation stay FP32 on the CUDA cores.
//
// Tile: 128 output rows (the MMA's M) x 32 output columns; radius R <= 24.
// One CTA per tile, 256 threads: every thread modulates a fixed set of
// (column, 8-row) items whose centred values stay in registers for the
// whole launch; thread 0 issues the MMAs; all threads move data out of TMEM.
// Every wait on the MMA completion barrier is bounded (spin_limit polls);
// if it runs out the CTA records BF_DEV_TIMEOUT, frees its TMEM and exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float k2PiHi = (float)kTwoPi;
constexpr float k2PiLo = (float)(kTwoPi - (double)(float)kTwoPi);
constexpr float kInv2Pi = (float)(1.0 / kTwoPi);

constexpr int TH = 128;           // output rows per tile = MMA M
constexpr int TW = 32;            // output columns per tile
constexpr int NT = 256;           // threads
constexpr int kMaxItems = 7;      // modulation items per thread (R <= 24)
constexpr int kCsStride = 36;     // fp32 words per row of the output cos / sin
constexpr int kTmemCols = 512;

__device__ __forceinline__ void phase_cs(float v, float om_hi, float om_lo, float& c, float& s)
{
    const float p = __fmul_rn(om_hi, v);
    float e = fmaf(om_hi, v, -p);
    e = fmaf(om_lo, v, e);
    const float q = rintf(__fmul_rn(p, kInv2Pi));
    float r = fmaf(-q, k2PiHi, p);
    r = fmaf(-q, k2PiLo, r);
    r = __fadd_rn(r, e);
    __sincosf(r, &s, &c);
}

template <bool kBF16>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if (kBF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}

// Eight values as one 16-byte row of a core matrix.
template <bool kBF16>
__device__ __forceinline__ void store_row8(unsigned char* dst, const float* v)
{
    *reinterpret_cast<uint4*>(dst) =
        make_uint4(pack2<kBF16>(v[0], v[1]), pack2<kBF16>(v[2], v[3]), pack2<kBF16>(v[4], v[5]),
                   pack2<kBF16>(v[6], v[7]));
}

// ---- PTX wrappers ---------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups along M / N.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;                     // descriptor version for tcgen05
    return d;                            // base offset 0, no swizzle
}

// Instruction descriptor, kind::f16: D = F32, A = B = F16 (0) or BF16 (1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the phase with the given parity; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit)
{
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// n (16 or 32) consecutive 32-bit TMEM columns of this thread's lane; the
// wait is in the same statement, so no use of v can be scheduled before it.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- geometry -------------------------------------------------------------

struct TcGeo {
    int R, RH, RW, RHp, RWp;
    uint32_t offA1, offB2, offP, offCS, bytes;   // byte offsets in dynamic smem
    uint32_t sboA1, sboB2, sboB1, sboA2, planeA2;
    __host__ __device__ TcGeo(int R_)
    {
        R = R_;
        RH = TH + 2 * R;
        RW = TW + 2 * R;
        RHp = (RH + 15) / 16 * 16;
        RWp = (RW + 15) / 16 * 16;
        sboA1 = (RHp / 8) * 128;       // A1: 128 rows (y) x RHp (r)
        sboB2 = (RWp / 8) * 128;       // B2: 32 rows (x) x RWp (j)
        sboB1 = (RHp / 8) * 128;       // B1: 4 RWp rows (p, j) x RHp (r)
        sboA2 = (RWp / 8) * 128;       // A2: per plane 128 rows (y) x RWp (j)
        planeA2 = TH * RWp * 2;
        const uint32_t a1 = TH * RHp * 2, b2 = TW * RWp * 2;
        const uint32_t b1 = 4u * RWp * RHp * 2, a2 = 4u * planeA2;
        const uint32_t p = b1 > a2 ? b1 : a2;
        offA1 = 0;
        offB2 = offA1 + a1;
        offP = offB2 + b2;
        offCS = offP + p;
        bytes = offCS + 2u * TH * kCsStride * 4 + 64;   // + barrier and TMEM slot
    }
};

template <bool kBF16>
__global__ void __launch_bounds__(NT, 1) k_fwd_tc(FwdArgs a, long long spin_limit,
                                                    unsigned* status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcGeo G(a.R);
    const int R = a.R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int by = blockIdx.y * TH, bx = blockIdx.x * TW;
    const int gy0 = by - R, gx0 = bx - R;
    float* cs = reinterpret_cast<float*>(smem + G.offCS);           // cos, then sin
    uint64_t* mbar_p = reinterpret_cast<uint64_t*>(smem + G.offCS + 2 * TH * kCsStride * 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar_p + 1);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t mbar = smem_u32(mbar_p);

    const int set = a.set_tile ? (by / a.set_tile) * a.sets_x + (bx / a.set_tile) : 0;
    const SetHdr hd = a.hdr[set];
    const float c0 = a.c0, inv_c0 = 1.0f / a.c0;

    if (hd.F < 0) {   // order above the cap: pass the image through
        for (int i = tid; i < TH * TW; i += NT) {
            const int gy = by + i / TW, gx = bx + i % TW;
            if (gy < a.H && gx < a.W)
                a.out[(size_t)gy * a.out_pitch + gx] = a.f[(size_t)gy * a.f_pitch + gx];
        }
        return;
    }

    // ---- TMEM, barrier
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tslot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) mbar_init(mbar);

    // ---- constant Toeplitz operands: A1 = Gv (128 x RHp), B2 = Gh (32 x RWp)
    for (int i = tid; i < TH * (G.RHp / 8); i += NT) {
        const int y = i / (G.RHp / 8), k8 = i % (G.RHp / 8);
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float t2[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int t = k8 * 8 + 2 * h + e - y;      // tap index r - y in [0, 2R]
                t2[e] = (t >= 0 && t <= 2 * R) ? a.taps[t] : 0.f;
            }
            w[h] = pack2<kBF16>(t2[0], t2[1]);
        }
        const uint32_t off = G.offA1 + (y / 8) * G.sboA1 + k8 * 128 + (y % 8) * 16;
        *reinterpret_cast<uint4*>(smem + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    for (int i = tid; i < TW * (G.RWp / 8); i += NT) {
        const int x = i / (G.RWp / 8), k8 = i % (G.RWp / 8);
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float t2[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int t = k8 * 8 + 2 * h + e - x;      // j - x in [0, 2R]
                t2[e] = (t >= 0 && t <= 2 * R) ? a.taps[t] : 0.f;
            }
            w[h] = pack2<kBF16>(t2[0], t2[1]);
        }
        const uint32_t off = G.offB2 + (x / 8) * G.sboB2 + k8 * 128 + (x % 8) * 16;
        *reinterpret_cast<uint4*>(smem + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }

    // ---- my modulation items: (column j, rows rb*8 .. rb*8+7) of the halo
    // region, j in [0, RWp), rb in [0, RHp/8); values kept in registers
    const int n_items = G.RWp * (G.RHp / 8);
    float fv[kMaxItems][8];
    uint32_t valid[kMaxItems];
#pragma unroll
    for (int t = 0; t < kMaxItems; ++t) {
        valid[t] = 0u;
        const int it = tid + t * NT;
        const int j = it % G.RWp, rb = it / G.RWp;
        const int gx = gx0 + j;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            fv[t][i] = 0.f;
            const int r = rb * 8 + i, gy = gy0 + r;
            if (it < n_items && j < G.RW && r < G.RH && gx >= 0 && gx < a.W && gy >= 0 &&
                gy < a.H) {
                fv[t][i] = __ldg(a.f + (size_t)gy * a.f_pitch + gx) - c0;
                valid[t] |= 1u << i;
            }
        }
    }

    // ---- epilogue ownership: lane quarter q = warp % 4 (TMEM lanes 32q..),
    // output row y = 32q + lane, columns x in [16h, 16h + 16), h = warp / 4
    const int q = warp & 3, hcol = warp >> 2;
    const int yl = 32 * q + lane;
    float num[16], den[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) num[i] = den[i] = 0.f;

    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t tD1 = tbase;                     // 4 RWp columns
    const uint32_t tD2 = tbase + 4 * G.RWp;         // 128 columns
    const uint32_t tlane = (uint32_t)(32 * q) << 16;

    const uint32_t idesc1 = idesc_f16(TH, 2 * G.RWp, kBF16);   // N = 2 RWp per MMA
    const uint32_t idesc2 = idesc_f16(TH, TW, kBF16);
    const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    const int K = hd.F + hd.z;
    uint32_t phase = 0;
    bool failed = false;

    for (int k = 0; k < K && !failed; ++k) {
        float om_hi = 0.f, om_lo = 0.f, Wk = hd.w0;
        if (k < hd.F) {
            const Pair p = pr[k];
            om_hi = p.om_hi;
            om_lo = p.om_lo;
            Wk = p.W;
        }

        // (1) modulate into B1 (K-major: rows (plane, j), K = r) and the
        //     FP32 cos / sin of the output pixels
#pragma unroll
        for (int t = 0; t < kMaxItems; ++t) {
            const int it = tid + t * NT;
            if (it >= n_items) break;
            const int j = it % G.RWp, rb = it / G.RWp;
            float cv[8], sv[8], av[8], bv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float c = 0.f, s = 0.f;
                if (valid[t] & (1u << i)) phase_cs(fv[t][i], om_hi, om_lo, c, s);
                const float pn = fv[t][i] * inv_c0;
                cv[i] = c;
                sv[i] = s;
                av[i] = pn * c;
                bv[i] = pn * s;
                const int y = rb * 8 + i - R, x = j - R;
                if (y >= 0 && y < TH && x >= 0 && x < TW) {
                    cs[y * kCsStride + x] = c;
                    cs[TH * kCsStride + y * kCsStride + x] = s;
                }
            }
            store_row8<kBF16>(smem + G.offP + ((0 * G.RWp + j) / 8) * G.sboB1 + rb * 128 +
                                  ((0 * G.RWp + j) % 8) * 16, av);
            store_row8<kBF16>(smem + G.offP + ((1 * G.RWp + j) / 8) * G.sboB1 + rb * 128 +
                                  ((1 * G.RWp + j) % 8) * 16, bv);
            store_row8<kBF16>(smem + G.offP + ((2 * G.RWp + j) / 8) * G.sboB1 + rb * 128 +
                                  ((2 * G.RWp + j) % 8) * 16, cv);
            store_row8<kBF16>(smem + G.offP + ((3 * G.RWp + j) / 8) * G.sboB1 + rb * 128 +
                                  ((3 * G.RWp + j) % 8) * 16, sv);
        }
        fence_async_smem();
        __syncthreads();

        // (2) vertical pass on the tensor cores: D1 = Gv * P^T
        if (tid == 0) {
            fence_after();
            for (int half = 0; half < 2; ++half) {
                const uint32_t nb = sbase + G.offP + (uint32_t)(half * 2 * G.RWp / 8) * G.sboB1;
                for (int ks = 0; ks < G.RHp / 16; ++ks) {
                    const uint64_t da = sdesc(sbase + G.offA1 + ks * 256, 128, G.sboA1);
                    const uint64_t db = sdesc(nb + ks * 256, 128, G.sboB1);
                    mma_f16(tD1 + half * 2 * G.RWp, da, db, idesc1, ks > 0);
                }
            }
            mma_commit(mbar);
        }
        bool ok = mbar_wait(mbar, phase, spin_limit);
        if (__syncthreads_or(!ok)) { failed = true; break; }
        phase ^= 1u;
        fence_after();

        // (3) D1 (FP32, TMEM) -> A2 (16-bit, shared, K-major: rows y, K = j)
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
            const int pl = 2 * hcol + pp;
            for (int c0c = 0; c0c < G.RWp; c0c += 32) {
                const bool two = c0c + 16 < G.RWp;
                float v[32];
                if (two) tmem_ld32(tD1 + tlane + pl * G.RWp + c0c, v);
                else tmem_ld16(tD1 + tlane + pl * G.RWp + c0c, v);
                const uint32_t off = G.offP + pl * G.planeA2 + (yl / 8) * G.sboA2 +
                                     (c0c / 8) * 128 + (yl % 8) * 16;
                store_row8<kBF16>(smem + off, v);
                store_row8<kBF16>(smem + off + 128, v + 8);
                if (two) {
                    store_row8<kBF16>(smem + off + 256, v + 16);
                    store_row8<kBF16>(smem + off + 384, v + 24);
                }
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();

        // (4) horizontal pass: D2_p = V_p * Gh^T for the four planes
        if (tid == 0) {
            fence_after();
            for (int pl = 0; pl < 4; ++pl) {
                for (int ks = 0; ks < G.RWp / 16; ++ks) {
                    const uint64_t da = sdesc(sbase + G.offP + pl * G.planeA2 + ks * 256, 128,
                                              G.sboA2);
                    const uint64_t db = sdesc(sbase + G.offB2 + ks * 256, 128, G.sboB2);
                    mma_f16(tD2 + pl * TW, da, db, idesc2, ks > 0);
                }
            }
            mma_commit(mbar);
        }
        ok = mbar_wait(mbar, phase, spin_limit);
        if (__syncthreads_or(!ok)) { failed = true; break; }
        phase ^= 1u;
        fence_after();

        // (5) demodulate and accumulate (eqs. (f1), (f2)): numerator planes,
        //     then denominator planes, 32 TMEM columns at a time
        {
            const float* crow = cs + yl * kCsStride + 16 * hcol;
            const float* srow = crow + TH * kCsStride;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                float va[16], vb[16];
                tmem_ld16(tD2 + tlane + (2 * part) * TW + 16 * hcol, va);
                tmem_ld16(tD2 + tlane + (2 * part + 1) * TW + 16 * hcol, vb);
                float* acc = part == 0 ? num : den;
#pragma unroll
                for (int i = 0; i < 16; i += 4) {
                    const float4 c4 = *reinterpret_cast<const float4*>(crow + i);
                    const float4 s4 = *reinterpret_cast<const float4*>(srow + i);
                    acc[i + 0] = fmaf(Wk, fmaf(c4.x, va[i + 0], s4.x * vb[i + 0]), acc[i + 0]);
                    acc[i + 1] = fmaf(Wk, fmaf(c4.y, va[i + 1], s4.y * vb[i + 1]), acc[i + 1]);
                    acc[i + 2] = fmaf(Wk, fmaf(c4.z, va[i + 2], s4.z * vb[i + 2]), acc[i + 2]);
                    acc[i + 3] = fmaf(Wk, fmaf(c4.w, va[i + 3], s4.w * vb[i + 3]), acc[i + 3]);
                }
            }
        }
        fence_before();
        __syncthreads();
    }

    if (failed) {
        if (tid == 0) atomicOr(status, kDevTimeout);
        // give the tensor core one more bounded chance to drain before freeing TMEM
        mbar_wait(mbar, phase, spin_limit);
    } else {
        // ---- normalise and write (den guard with the FP32 clipped Gaussian mass)
        const int gy = by + yl;
        if (gy < a.H) {
            float rmass = 0.f;
            for (int t = -R; t <= R; ++t)
                if (gy + t >= 0 && gy + t < a.H) rmass += a.taps[t + R];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int gx = bx + 16 * hcol + i;
                if (gx >= a.W) continue;
                float cmass = 0.f;
                for (int t = -R; t <= R; ++t)
                    if (gx + t >= 0 && gx + t < a.W) cmass += a.taps[t + R];
                float v;
                if (den[i] > kGuard * rmass * cmass) {
                    v = __fdiv_rn(num[i], den[i]) * c0 + c0;
                } else {
                    v = a.f[(size_t)gy * a.f_pitch + gx];
                    atomicAdd(a.n_guarded, 1ull);
                }
                a.out[(size_t)gy * a.out_pitch + gx] = v;
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tbase), "r"(kTmemCols) : "memory");
    }
}

template <bool kBF16>
cudaError_t launch_t(const FwdArgs& a, long long spin, unsigned* status, cudaStream_t s)
{
    const TcGeo G(a.R);
    cudaError_t e = cudaFuncSetAttribute(k_fwd_tc<kBF16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G.bytes);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    k_fwd_tc<kBF16><<<grid, NT, G.bytes, s>>>(a, spin, status);
    return cudaGetLastError();
}

}  // namespace

// Largest R the tensor-core kernel takes (shared memory, TMEM columns and
// the per-thread item count all fit).
int fwd_tc_max_radius()
{
    int best = -1;
    for (int R = 0; R <= 64; ++R) {
        const TcGeo G(R);
        const int items = G.RWp * (G.RHp / 8);
        if (G.bytes <= 227 * 1024 && 4 * G.RWp + 4 * TW <= kTmemCols &&
            items <= kMaxItems * NT && 2 * G.RWp <= 256)
            best = R;
        else
            break;
    }
    return best;
}

void fwd_tc_tile(int* th, int* tw)
{
    *th = TH;
    *tw = TW;
}

cudaError_t launch_fwd_tc(const FwdArgs& a, bool bf16, long long spin, unsigned* status,
                          cudaStream_t s)
{
    if (a.R > fwd_tc_max_radius()) return cudaErrorInvalidValue;
    return bf16 ? launch_t<true>(a, spin, status, s) : launch_t<false>(a, spin, status, s);
}

}  // namespace bf
