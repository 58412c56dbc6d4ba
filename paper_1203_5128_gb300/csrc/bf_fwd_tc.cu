// K3-tc: fused SHIFTABLE-BF forward with FP16 / BF16 planes on the 5th-gen
// tensor cores (tcgen05, accumulators in TMEM), warp-specialised and
// pipelined across the terms of phi_eps.
//
// Same method as K3 (Sec. 1.2, eqs. (f1)-(f2) with phi_eps of eq. (approx)):
// per kept pair, modulate, Gaussian-filter the four planes, demodulate and
// accumulate num / den.  The spatial Gaussian of a 128 x 32 output tile is
// two dense products with constant banded matrices, the shape tcgen05.mma
// executes:
//
//   vertical   D1[m, (p, j)] = sum_r Gv[m, r] * P[(p, j), r]     (M = 128)
//   horizontal D2[m, (p, n)] = sum_j V_p[m, j] * Gh[n, j]        (per plane p)
//
// P holds the four modulated planes of the tile + halo (K-major, r fastest);
// V_p is D1 converted to 16 bits by the threads (TMEM -> registers -> shared,
// K-major with j fastest: no transpose).  Output rows and columns are taken
// in reverse order (m = 127 - y, n = 31 - x), which makes Gv[m, r] =
// g(r + m - 127 - R) and Gh[n, j] = g(j + n - 31 - R) depend on the sum of
// the indices: every 8 x 8 core matrix of such a Hankel matrix depends only
// on the sum of its block indices, so one row of distinct core matrices,
// read with both descriptor strides equal to 128 bytes, stands for the whole
// matrix (6 KB instead of 50 KB of shared memory).
//
// Roles (512 threads, one CTA per SM):
//   warps 0-3   TMEM lane quarters: D1 -> V (shared, one TMEM wait per plane),
//               then D2 -> demodulate into num / den (their output row, kept
//               in the 64 TMEM columns after D2), normalise, store;
//   warps 4-14  modulate the halo planes of pair k+1 while the tensor core
//               and warps 0-3 work on pair k;
//   warp 15     allocates TMEM, issues the MMAs, frees TMEM.
// Eleven modulation warps split the 80 x 22 (column, 8-row block) items of the
// R = 24 halo evenly, five per thread; with 16 warps the SM's register file
// gives each thread 128 registers.
// The conversion of D1 signals each plane of A2 on a barrier of its own, so
// the horizontal product of plane p runs while plane p + 1 is converted.
// Handshakes are mbarriers; every wait is bounded (spin_limit polls) and a
// wait that runs out sets BF_DEV_TIMEOUT, tells the other roles to stop,
// lets the tensor core drain (again bounded) and frees TMEM.
//
// The planes are 16-bit, so their phases need no more than FP32 single
// products: theta = (omega c0) * ((f - c0) / c0), with the same rounding at
// the halo pixel (modulation) and at the output pixel (demodulation).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int TH = 128;          // output rows per tile = MMA M
constexpr int TW = 32;           // output columns per tile
constexpr int kEpiWarps = 4;
constexpr int kModWarps = 11;
constexpr int NT = (kEpiWarps + kModWarps + 1) * 32;   // 512
constexpr int kModThreads = kModWarps * 32;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kMaxItems = 5;     // modulation items per thread (R <= 24)
constexpr int kTmemCols = 512;
constexpr int kPnStride = TW + 1;   // fp32 words per row of the output pixels' scaled f

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

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase of the given parity.  Returns false when the
// CTA is stopping: this wait ran out (it then raises the stop flag) or
// another role raised it.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit,
                                          volatile int* stop)
{
    for (long long i = 0;; ++i) {
        if (mbar_try(mbar, parity)) return true;
        if ((i & 63) == 63) {
            if (*stop) return false;
            if (i >= limit) {
                *stop = 1;
                return false;
            }
        }
    }
}

// mbar_wait taken by a whole warp: true only when every lane's wait
// succeeded, so that the warp leaves its loop as one and the warp-wide
// (.sync.aligned) TMEM instructions after the wait always run with all lanes.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t mbar, uint32_t parity, long long limit,
                                               volatile int* stop)
{
    return __all_sync(0xffffffffu, mbar_wait(mbar, parity, limit, stop));
}

// TMEM loads of this thread's lane; the wait is in the same statement, so no
// use of the outputs can be scheduled before it.
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

// Eight columns from each of four TMEM column ranges (one wait).

// TMEM loads of this thread's lane, several per wait (outputs only after it)
__device__ __forceinline__ void tmem_ld_48(uint32_t t0, uint32_t t1, float* v)
{
    uint32_t r[48];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%48];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%49];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
        : "r"(t0), "r"(t1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 48; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_64(uint32_t t0, float* v)
{
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(t0)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_80(uint32_t t0, uint32_t t1, float* v)
{
    uint32_t r[80];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%80];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%64,%65,%66,%67,%68,%69,%70,%71,%72,%73,%74,%75,%76,%77,%78,%79}, [%81];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63]), "=r"(r[64]), "=r"(r[65]), "=r"(r[66]), "=r"(r[67]), "=r"(r[68]), "=r"(r[69]), "=r"(r[70]), "=r"(r[71]), "=r"(r[72]), "=r"(r[73]), "=r"(r[74]), "=r"(r[75]), "=r"(r[76]), "=r"(r[77]), "=r"(r[78]), "=r"(r[79])
        : "r"(t0), "r"(t1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 80; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_6x8(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, uint32_t t4, uint32_t t5, float* v)
{
    uint32_t r[48];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%48];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%49];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%50];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%51];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32,%33,%34,%35,%36,%37,%38,%39}, [%52];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40,%41,%42,%43,%44,%45,%46,%47}, [%53];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5)
        : "memory");
#pragma unroll
    for (int i = 0; i < 48; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_2x32(uint32_t t0, uint32_t t1, float* v)
{
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(t0), "r"(t1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// Store 8 columns of this thread's lane (completion: tcgen05.wait::st).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                   "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])),
                   "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// The NCH * 16 columns of one plane of D1 in this thread's lane, one wait.
template <int NCH>
__device__ __forceinline__ void tmem_ld_plane(uint32_t taddr, float* v)
{
    if constexpr (NCH == 2) tmem_ld32(taddr, v);
    else if constexpr (NCH == 3) tmem_ld_48(taddr, taddr + 32, v);
    else if constexpr (NCH == 4) tmem_ld_64(taddr, v);
    else tmem_ld_80(taddr, taddr + 64, v);
}


// ---- geometry -------------------------------------------------------------

struct TcGeo {
    int R, RH, RW, RHp, RWp;
    int nA1, nB2;                                   // Hankel core matrices
    uint32_t offA1, offB2, offB1, offA2, offPn, offBar, bytes;
    uint32_t sboB1, sboA2, planeA2;
    __host__ __device__ TcGeo(int R_)
    {
        R = R_;
        RH = TH + 2 * R;
        RW = TW + 2 * R;
        RHp = (RH + 15) / 16 * 16;
        RWp = (RW + 15) / 16 * 16;
        nA1 = TH / 8 + RHp / 8 - 1;
        nB2 = TW / 8 + RWp / 8 - 1;
        sboB1 = (RHp / 8) * 128;       // B1: 4 RWp rows (plane, j) x RHp (r)
        sboA2 = (RWp / 8) * 128;       // A2: per plane 128 rows (m) x RWp (j)
        planeA2 = TH * RWp * 2;
        offA1 = 0;
        offB2 = offA1 + nA1 * 128;
        offB1 = offB2 + nB2 * 128;
        offA2 = offB1 + 4u * RWp * RHp * 2;
        offPn = offA2 + 4u * planeA2;
        offBar = offPn + TH * kPnStride * 4;
        bytes = offBar + 96;
    }
};

// barrier slots (8 bytes each) after the operand buffers
// (kBarNever: a barrier no thread arrives on, waited for only when a test
// asks the kernel to run out a bounded wait; bf_test_stall)
enum { kBarB1Full = 0, kBarC1, kBarA2Full, kBarA2F1, kBarA2F2, kBarA2F3, kBarC2, kBarD2Free,
       kBarNever, kNumBars };
static_assert(8 * kNumBars + 12 <= 96, "barrier slots, TMEM slot and stop flag fit the tail");

// Bound of the waits that let committed MMAs finish before a stopping CTA
// frees its TMEM: independent of spin_limit (MMAs finish within microseconds;
// this bound is seconds of polls), so that a short spin_limit never frees
// TMEM under an MMA in flight.
constexpr long long kDrainLimit = 1ll << 24;

template <bool kBF16, int NCH>
__global__ void __launch_bounds__(NT, 1) k_fwd_tc(FwdArgs a, long long spin_limit,
                                                    unsigned* status)
{
    constexpr int RWp = NCH * 16;
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcGeo G(a.R);
    const int R = a.R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int by = (blockIdx.y + a.y_tile0) * TH, bx = blockIdx.x * TW;
    const int gy0 = by - R, gx0 = bx - R;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + G.offBar;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + G.offBar + 8 * kNumBars);
    volatile int* stop = reinterpret_cast<volatile int*>(smem + G.offBar + 8 * kNumBars + 8);
    auto bar = [&](int i) { return bar0 + 8u * i; };

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

    // ---- set-up: TMEM, barriers, constant Hankel operands
    if (warp == kEpiWarps + kModWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tslot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar(kBarB1Full), kModThreads);
        mbar_init(bar(kBarC1), 1);
        for (int pl = 0; pl < 4; ++pl) mbar_init(bar(kBarA2Full + pl), kEpiThreads);
        mbar_init(bar(kBarC2), 1);
        mbar_init(bar(kBarD2Free), kEpiThreads);
        mbar_init(bar(kBarNever), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *stop = 0;
    }
    // Gv (rows reversed): core matrix d holds g(8d + i + e - (TH-1) - R)
    for (int i = tid; i < G.nA1 * 8; i += NT) {
        const int d = i / 8, row = i % 8;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int t = 8 * d + row + e - (TH - 1);    // r - y, tap index in [0, 2R]
            v[e] = (t >= 0 && t <= 2 * R) ? a.taps[t] : 0.f;
        }
        store_row8<kBF16>(smem + G.offA1 + d * 128 + row * 16, v);
    }
    // Gh (columns reversed): core matrix d holds g(8d + i + e - (TW-1) - R)
    for (int i = tid; i < G.nB2 * 8; i += NT) {
        const int d = i / 8, row = i % 8;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int t = 8 * d + row + e - (TW - 1);    // j - x
            v[e] = (t >= 0 && t <= 2 * R) ? a.taps[t] : 0.f;
        }
        store_row8<kBF16>(smem + G.offB2 + d * 128 + row * 16, v);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t tD1 = tbase;                  // 4 RWp columns
    const uint32_t tD2 = tbase + 4 * RWp;        // 4 x 32 columns
    const Pair* pr = a.pairs + (size_t)set * a.cap_pairs;
    const int K = hd.F + hd.z;

    if (warp >= kEpiWarps && warp < kEpiWarps + kModWarps) {
        // ================= modulation warps =================
        const int mt = tid - kEpiThreads;
        const int n_items = RWp * (G.RHp / 8);
        float pn[kMaxItems][8];
        uint32_t valid[kMaxItems];
#pragma unroll
        for (int t = 0; t < kMaxItems; ++t) {
            valid[t] = 0u;
            const int it = mt + t * kModThreads;
            const int j = it % RWp, rb = it / RWp;
            const int gx = gx0 + j;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                pn[t][i] = 0.f;
                const int r = rb * 8 + i, gy = gy0 + r;
                if (it < n_items && j < G.RW && r < G.RH && gx >= 0 && gx < a.W && gy >= 0 &&
                    gy < a.H) {
                    const float f = __ldg(a.f + (size_t)gy * a.f_pitch + gx);
                    pn[t][i] = __fmul_rn(__fsub_rn(f, c0), inv_c0);
                    valid[t] |= 1u << i;
                }
            }
        }
        for (int k = 0; k < K; ++k) {
            const float wc = k < hd.F ? __fmul_rn(pr[k].om_hi, c0) : 0.f;
            if (k > 0 && !mbar_wait(bar(kBarC1), (k - 1) & 1, spin_limit, stop)) break;
#pragma unroll
            for (int t = 0; t < kMaxItems; ++t) {
                const int it = mt + t * kModThreads;
                if (it >= n_items) break;
                const int j = it % RWp, rb = it / RWp;
                float cv[8], sv[8], av[8], bv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float s, c;
                    __sincosf(__fmul_rn(wc, pn[t][i]), &s, &c);
                    const bool v = (valid[t] >> i) & 1u;
                    c = v ? c : 0.f;
                    s = v ? s : 0.f;
                    cv[i] = c;
                    sv[i] = s;
                    av[i] = pn[t][i] * c;
                    bv[i] = pn[t][i] * s;
                }
                unsigned char* b1 = smem + G.offB1 + rb * 128;
                store_row8<kBF16>(b1 + ((0 * RWp + j) / 8) * G.sboB1 + ((0 * RWp + j) % 8) * 16, av);
                store_row8<kBF16>(b1 + ((1 * RWp + j) / 8) * G.sboB1 + ((1 * RWp + j) % 8) * 16, bv);
                store_row8<kBF16>(b1 + ((2 * RWp + j) / 8) * G.sboB1 + ((2 * RWp + j) % 8) * 16, cv);
                store_row8<kBF16>(b1 + ((3 * RWp + j) / 8) * G.sboB1 + ((3 * RWp + j) % 8) * 16, sv);
            }
            fence_async_smem();
            mbar_arrive(bar(kBarB1Full));
        }
    } else if (warp == kEpiWarps + kModWarps) {
        // ================= MMA issue (one thread) =================
        if (lane == 0) {
            const uint32_t idesc1 = idesc_f16(TH, 2 * RWp, kBF16);
            const uint32_t idesc2 = idesc_f16(TH, TW, kBF16);
            int issued1 = 0, issued2 = 0;
            // a test's stall: wait (bounded) for a barrier nothing arrives on
            if (a.stall_test) mbar_wait(bar(kBarNever), 0, spin_limit, stop);
            for (int k = 0; k < K; ++k) {
                if (!mbar_wait(bar(kBarB1Full), k & 1, spin_limit, stop)) break;
                fence_after();
                // consecutive MMAs go to different accumulators, so that no
                // MMA waits on the previous one's accumulation
                for (int ks = 0; ks < G.RHp / 16; ++ks) {
                    const uint64_t da = sdesc(sbase + G.offA1 + ks * 256, 128, 128);
                    for (int half = 0; half < 2; ++half) {
                        const uint32_t nb =
                            sbase + G.offB1 + (uint32_t)(half * 2 * RWp / 8) * G.sboB1;
                        const uint64_t db = sdesc(nb + ks * 256, 128, G.sboB1);
                        mma_f16(tD1 + half * 2 * RWp, da, db, idesc1, ks > 0);
                    }
                }
                mma_commit(bar(kBarC1));
                ++issued1;
                if (k > 0 && !mbar_wait(bar(kBarD2Free), (k - 1) & 1, spin_limit, stop)) break;
                // each plane's horizontal product as soon as that plane of A2 is written
                bool planes_ok = true;
                for (int pl = 0; pl < 4; ++pl) {
                    if (!mbar_wait(bar(kBarA2Full + pl), k & 1, spin_limit, stop)) { planes_ok = false; break; }
                    fence_after();
#pragma unroll
                    for (int ks = 0; ks < NCH; ++ks) {
                        const uint64_t db = sdesc(sbase + G.offB2 + ks * 256, 128, 128);
                        const uint64_t da = sdesc(sbase + G.offA2 + pl * G.planeA2 + ks * 256, 128,
                                                  G.sboA2);
                        mma_f16(tD2 + pl * TW, da, db, idesc2, ks > 0);
                    }
                }
                if (!planes_ok) {
                    mma_commit(bar(kBarC2));      // so that the drain below waits for them
                    ++issued2;
                    break;
                }
                mma_commit(bar(kBarC2));
                ++issued2;
            }
            if (*stop) {
                // let every committed MMA finish before TMEM is freed (bounded)
                volatile int never = 0;
                if (issued1) mbar_wait(bar(kBarC1), (issued1 - 1) & 1, kDrainLimit, &never);
                if (issued2) mbar_wait(bar(kBarC2), (issued2 - 1) & 1, kDrainLimit, &never);
            }
        }
        __syncwarp();
    } else {
        // ================= epilogue warps (TMEM lanes 32 q ..) =================
        const int q = warp;
        const int m = 32 * q + lane;              // MMA row = TMEM lane
        const int y = TH - 1 - m;                 // output row of this thread
        const int gy = by + y;
        const uint32_t tl = (uint32_t)(32 * q) << 16;
        // centred, scaled f of my outputs, in shared memory (row m, padded)
        float* pno = reinterpret_cast<float*>(smem + G.offPn) + m * kPnStride;
#pragma unroll
        for (int x = 0; x < TW; ++x) {
            const int gx = bx + x;
            pno[x] = (gy < a.H && gx < a.W)
                         ? __fmul_rn(__fsub_rn(__ldg(a.f + (size_t)gy * a.f_pitch + gx), c0), inv_c0)
                         : 0.f;
        }
        // num / den of my row in TMEM columns tND .. tND + 63 (32 each)
        const uint32_t tND = tbase + 4 * RWp + 4 * TW + tl;
        {
            float z[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) z[e] = 0.f;
#pragma unroll
            for (int q8 = 0; q8 < 8; ++q8) tmem_st8(tND + 8 * q8, z);
            tmem_wait_st();
        }
        bool ok = true;
        for (int k = 0; k < K && ok; ++k) {
            float wc = 0.f, Wk = hd.w0;
            if (k < hd.F) {
                const Pair p = pr[k];
                wc = __fmul_rn(p.om_hi, c0);
                Wk = p.W;
            }
            // D1 ready: convert my row of each plane to 16 bits (A2, K-major)
            if (!mbar_wait_warp(bar(kBarC1), k & 1, spin_limit, stop)) { ok = false; break; }
            fence_after();
            unsigned char* a2row = smem + G.offA2 + (m / 8) * G.sboA2 + (m % 8) * 16;
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) {
                float v[NCH * 16];
                tmem_ld_plane<NCH>(tD1 + tl + pl * RWp, v);
                unsigned char* dst = a2row + pl * G.planeA2;
#pragma unroll
                for (int b8 = 0; b8 < 2 * NCH; ++b8) store_row8<kBF16>(dst + b8 * 128, v + 8 * b8);
                fence_async_smem();
                fence_before();
                mbar_arrive(bar(kBarA2Full + pl));
            }
            // D2 ready: demodulate (eqs. (f1), (f2)); TMEM column n is x = 31 - n
            if (!mbar_wait_warp(bar(kBarC2), k & 1, spin_limit, stop)) { ok = false; break; }
            fence_after();
#pragma unroll
            for (int cb = 0; cb < TW / 8; ++cb) {
                float v[48];
                tmem_ld_6x8(tD2 + tl + 0 * TW + 8 * cb, tD2 + tl + 1 * TW + 8 * cb,
                            tD2 + tl + 2 * TW + 8 * cb, tD2 + tl + 3 * TW + 8 * cb,
                            tND + 8 * cb, tND + TW + 8 * cb, v);
                float nn[8], dd[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int x = TW - 1 - (8 * cb + e);
                    float s, c;
                    __sincosf(__fmul_rn(wc, pno[x]), &s, &c);
                    nn[e] = fmaf(Wk, fmaf(c, v[e], s * v[8 + e]), v[32 + e]);
                    dd[e] = fmaf(Wk, fmaf(c, v[16 + e], s * v[24 + e]), v[40 + e]);
                }
                tmem_st8(tND + 8 * cb, nn);
                tmem_st8(tND + TW + 8 * cb, dd);
            }
            tmem_wait_st();
            fence_before();
            mbar_arrive(bar(kBarD2Free));
        }
        tmem_wait_st();
        float num[TW], den[TW];
        {
            float nd[2 * TW];
            tmem_ld_2x32(tND, tND + TW, nd);
            // TMEM column 8 cb + e holds output x = 31 - (8 cb + e)
#pragma unroll
            for (int n = 0; n < TW; ++n) {
                num[TW - 1 - n] = nd[n];
                den[TW - 1 - n] = nd[TW + n];
            }
        }
        if (ok && gy < a.H) {
            // normalise with the guard (FP32 clipped Gaussian mass) and store
            const float full = full_mass(a.taps, R);
            const float rmass = clipped_mass(a.taps, R, gy, a.H, full);
            // outputs whose den is under fix_kappa of their mass: the 16-bit
            // rounding is amplified by mass / den there, so the FP32 recheck
            // writes them (and applies the guard); they are only marked in the
            // unrolled loop and listed after it, which keeps the loop small
            // (no list when the recheck is off: then nothing is listed, not
            // even an output whose den is negative)
            const float kap = a.fix_list ? a.fix_kappa : -INFINITY;
            uint32_t listed = 0u;
#pragma unroll
            for (int x = 0; x < TW; ++x) {
                const int gx = bx + x;
                if (gx >= a.W) continue;
                const float cmass = clipped_mass(a.taps, R, gx, a.W, full);
                float v;
                if (den[x] < kap * rmass * cmass) {
                    listed |= 1u << x;
                    v = a.f[(size_t)gy * a.f_pitch + gx];
                } else if (den[x] > kGuard * rmass * cmass) {
                    v = __fdiv_rn(num[x], den[x]) * c0 + c0;
                } else {
                    v = a.f[(size_t)gy * a.f_pitch + gx];
                    atomicAdd(a.n_guarded, 1ull);
                }
                a.out[(size_t)gy * a.out_pitch + gx] = v;
            }
            while (listed) {
                const int x = __ffs(listed) - 1;
                listed &= listed - 1u;
                a.fix_list[(size_t)set * a.fix_cap + atomicAdd(a.fix_count + set, 1u)] =
                    (unsigned)gy * (unsigned)a.W + (unsigned)(bx + x);
            }
        }
    }

    fence_before();
    __syncthreads();
    if (tid == 0 && *stop) atomicOr(status, kDevTimeout);
    if (warp == kEpiWarps + kModWarps) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tbase), "r"(kTmemCols) : "memory");
    }
}

template <bool kBF16, int NCH>
cudaError_t launch_t(const FwdArgs& a, long long spin, unsigned* status, cudaStream_t s)
{
    const TcGeo G(a.R);
    cudaError_t e = cudaFuncSetAttribute(k_fwd_tc<kBF16, NCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G.bytes);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, a.y_tiles > 0 ? a.y_tiles : (a.H + TH - 1) / TH);
    k_fwd_tc<kBF16, NCH><<<grid, NT, G.bytes, s>>>(a, spin, status);
    return cudaGetLastError();
}

template <bool kBF16>
cudaError_t launch_nch(const FwdArgs& a, long long spin, unsigned* status, cudaStream_t s)
{
    switch (TcGeo(a.R).RWp / 16) {
    case 2: return launch_t<kBF16, 2>(a, spin, status, s);
    case 3: return launch_t<kBF16, 3>(a, spin, status, s);
    case 4: return launch_t<kBF16, 4>(a, spin, status, s);
    case 5: return launch_t<kBF16, 5>(a, spin, status, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// Largest R the tensor-core kernel takes: shared memory, TMEM columns, the
// per-thread item count and the N of one vertical MMA all fit.
int fwd_tc_max_radius()
{
    int best = -1;
    for (int R = 0; R <= 64; ++R) {
        const TcGeo G(R);
        const int items = G.RWp * (G.RHp / 8);
        if (G.bytes <= 227 * 1024 && 4 * G.RWp + 4 * TW <= kTmemCols &&
            items <= kMaxItems * kModThreads && 2 * G.RWp <= 256 && G.RWp / 16 <= 5)
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
    return bf16 ? launch_nch<true>(a, spin, status, s) : launch_nch<false>(a, spin, status, s);
}

}  // namespace bf
