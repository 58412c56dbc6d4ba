// Internal declarations shared by the CUDA translation units of libbf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bf.h"

namespace bf {
struct SetHdr;
struct Pair;
}

// A plan: the sizes, options and device workspace of one image shape.
struct bf_plan_s {
    int H, W, R;
    double sigma_s, sigma_r, eps;
    bf_options opt;
    int device;
    int n_sets, sets_x, sets_y, set_tile;
    int n_cap, cap_pairs;
    float c0;
    int th, tw;
    unsigned* d_T;
    bf::SetHdr* d_hdr;
    bf::Pair* d_pairs;
    float* d_taps;
    float* h_taps;          // host copy of the 2R+1 taps
    double* d_logfact;
    unsigned* d_status;
    unsigned long long* d_nguard;
    float* d_hin;
    float* d_hout;
    float* d_bwd;            // backward scratch (out, den), allocated on first use
    int executed;
    cudaStream_t last;
    int yvv_C, yvv_passes;   // recursive filter: terms per pass (8 or 16), passes
    int yvv_G;               // recursive filter: passes per launch (32 / C)
    float4* d_yvv_P;         // recursive filter: row-filtered planes [H][W][32]
    float4* d_yvv_S;         // recursive filter: row states [H][ceil(W/8)][3][32]
    float2* d_yvv_nd;        // recursive filter: (num, den) partials [G][H][W]
    float* d_yvv_mass;       // recursive filter: mass_y[H] then mass_x[W]
    float* d_sep_P;          // two-pass FIR: row-filtered planes of sep_nk terms
    float2* d_sep_nd;        // two-pass FIR: (num, den) partial
    int sep_nk, sep_Wp;
    int timing;              // record events around the kernels
    int n_timed;
    cudaEvent_t* ev;         // 4 per recorded execute
    unsigned* d_mm;          // raised polynomial: codes of max f and max -f per set
    int patch_p;             // non-local means: patch pixels (0: the bilateral filter)
    int stall_test;          // bf_test_stall
    int patch_uy[9], patch_ux[9];
    unsigned* d_fix;         // 16-bit recheck: listed pixels (y * W + x), H * W slots
    unsigned* d_fixcnt;      // 16-bit recheck: list lengths, one per parameter set
    unsigned* d_fixscan;     // 16-bit recheck: their offsets (n_sets + 1 per launch;
                             // concurrent row bands take disjoint ranges)
    unsigned fix_cap;        // 16-bit recheck: list slots per set
    int n_fixcnt;
    cudaStream_t hst[5];     // banded host path: copy in, compute (2), copy out, recheck
    cudaEvent_t* hev;        // banded host path: fork, clear, join, then per band in / done
    int n_hev;
};

namespace bf {

// One parameter set (Algorithm 2, steps 3-5) as the forward kernels read it.
// F folded frequency pairs (n and N-n, weight 2 w_n) follow in the pair
// table; z = 1 when the zero frequency n = N/2 is kept (weight w0).
// F < 0 marks a set whose N exceeded the plan's cap.
struct SetHdr {
    int N, M, F, z;
    float w0, T, pad0, pad1;
};

// Pair k of a set: omega = (2n - N) / (sqrt(N) sigma_r) > 0 split into an
// FP32 head and tail (hi + lo), and the folded weight W = 2 w_n.
struct Pair {
    float om_hi, om_lo, W, pad;
};

// Clipped Gaussian mass along one axis (the denominator guard's
// (g * 1_Omega) factor): the sum of taps[t + R] over the t with 0 <= i + t < n,
// added in increasing t.  `full` is the same sum over every t (the same
// additions in the same order), which is the value at every coordinate at
// least R from both ends, so only coordinates near the border loop.
__device__ __forceinline__ float clipped_mass(const float* taps, int R, int i, int n, float full)
{
    if (i - R >= 0 && i + R < n) return full;
    float m = 0.f;
    for (int t = -R; t <= R; ++t)
        if (i + t >= 0 && i + t < n) m += taps[t + R];
    return m;
}
__device__ __forceinline__ float full_mass(const float* taps, int R)
{
    float m = 0.f;
    for (int t = -R; t <= R; ++t) m += taps[t + R];
    return m;
}

// Device status bits (mirrors BF_DEV_* of bf.h).
constexpr unsigned kDevOrder = 1u << 0;
constexpr unsigned kDevTimeout = 1u << 1;
constexpr unsigned kDevBadWork = 1u << 2;

// Denominator guard (the paper is silent): where den <= kGuard * (g * 1_Omega)
// the output is f(x).
constexpr float kGuard = 1e-6f;

// ---- launchers (each in its own translation unit) ------------------------

// K1: local range r(x) = max(M(x) - f(x), f(x) - m(x)) reduced to one
// non-negative float per T-set (atomicMax on the bit pattern).  Tbits must be
// zeroed first.  set_tile == 0: one set for the whole image.
// by0 / nby: the 64-row block rows of the launch (nby = 0: all).
cudaError_t launch_local_range(const float* f, size_t pitch, int H, int W, int R,
                               int set_tile, int sets_x, unsigned* Tbits, cudaStream_t s,
                               int by0 = 0, int nby = 0);

// Largest R whose K1 staging fits in shared memory.
int range_max_radius();

// K1 as images: windowed max and min (testing entry point).
cudaError_t launch_maxmin(const float* f, size_t pitch, int H, int W, int R, float* Mx,
                          float* mn, cudaStream_t s);

// K2: N, M and the pair table for every set from its T.
struct ParamsArgs {
    const float* T;        // [n_sets]
    int n_sets;
    double sigma_r, eps, value_range;
    int rule;
    int n_cap;             // largest N the pair table can hold
    int cap_pairs;         // pairs per set in the table
    const double* logfact; // log(k!) for k = 0..n_cap (host lgamma)
    double ln2;
    SetHdr* hdr;
    Pair* pairs;
    unsigned* status;
    int set0 = 0;          // first set of the launch (block b takes set set0 + b)
};
// K2 over sets set0 .. set0 + n - 1 (n = 0: all sets).
cudaError_t launch_params(const ParamsArgs& a, cudaStream_t s, int n = 0);

// K1 + K2 fused for T-tiles of side set_tile (a multiple of 64): one CTA
// per T-tile computes its exact T (written to Tbits[set]) and its parameter
// set; sets set0 .. set0 + n_sets - 1.  tile_params_ok: the staging fits.
bool tile_params_ok(int R, int set_tile, int n_cap);
cudaError_t launch_tile_params(const float* f, size_t pitch, int H, int W, int R, int set_tile,
                               int sets_x, int set0, int n_sets, unsigned* Tbits,
                               const ParamsArgs& pa, cudaStream_t s);

// K3 (FP32 planes, FIR): fused modulate / filter / demodulate / normalise.
struct FwdArgs {
    int y_tile0 = 0;        // first row of output tiles of the launch
    int y_tiles = 0;        // rows of output tiles (0: the whole image)
    const float* f;
    size_t f_pitch;
    float* out;
    size_t out_pitch;
    int H, W, R;
    const float* taps;      // 2R+1 FP32 spatial taps g(k)
    const SetHdr* hdr;
    const Pair* pairs;
    int cap_pairs;
    int set_tile;           // 0: single set; else T-tile side
    int sets_x;
    float c0;               // centring constant (value_range / 2)
    unsigned long long* n_guarded;
    float* den_out;         // optional: den per pixel (backward)
    size_t den_pitch;
    const float* h_taps;    // host copy of taps (null: shared-memory taps only)
    // two-pass workspace for radii beyond the fused tall tile (null: none)
    float* sep_P;           // [nk][4][H][sep_Wp] row-filtered planes
    float2* sep_nd;         // [H][W] (num, den) partial
    int sep_nk, sep_Wp, sep_cap_terms;
    // 16-bit planes: outputs with den < fix_kappa * mass are appended to
    // their set's list (y * W + x; set s owns fix_list[s * fix_cap ..], its
    // length in fix_count[s]) for the FP32 recheck instead of being final
    unsigned* fix_list = nullptr;
    unsigned* fix_count = nullptr;
    unsigned fix_cap = 0;
    float fix_kappa = 0.f;
    int stall_test = 0;     // K3-tc: run out a bounded wait (bf_test_stall)
    int box_rs = 0;         // box spatial filter: FP32 planes by exact running sums
    int box = 0;            // box spatial filter (unit taps): sliding sums in the tall FIR
};

// FP32 recheck of listed outputs of a 16-bit-plane forward: the direct sum
// of eq. (BF) with phi_eps of the pixel's own parameter set.
struct FixArgs {
    const float* f;
    size_t f_pitch;
    float* out;
    size_t out_pitch;
    int H, W, R;
    const float* taps;      // 2R+1 device taps
    const SetHdr* hdr;
    const Pair* pairs;
    int cap_pairs;
    int set_tile;           // 0: single set; else T-tile side
    int sets_x;
    double sigma_r;
    const unsigned* list;   // pixels y * W + x, set s from list[s * fix_cap]
    const unsigned* count;  // list length per set (device)
    unsigned fix_cap;
    unsigned long long* n_guarded;
    int set0;               // first set of the launch
    int ntab;               // floats of phi_eps table a CTA holds (four per interval)
    unsigned* scan;         // n_sets + 1 offsets (scratch)
};
int fixup_table_entries(int n_cap);
// The recheck of what a 16-bit forward with arguments fa lists (bf_api.cu).
FixArgs fixup_args(bf_plan_s* p, const FwdArgs& fa);
// FP32 recheck of the listed outputs of sets set0 .. set0 + n_sets - 1.
cudaError_t launch_fixup(const FixArgs& a, int n_sets, cudaStream_t s);

// Raised-polynomial range kernel (eq. (RPconv)): per-set range of f, then
// N, centre, half-range, beta and the Chebyshev nodes, then the fused tile.
struct PolyParamsArgs {
    const unsigned* mm;     // per set: codes of max f and max -f (null: fixed T)
    int n_sets;
    double sigma_r, t_fixed, value_range;
    int n_cap;              // largest N the node table holds
    int cap_nodes;          // node entries per set (2 n_cap + 1)
    SetHdr* hdr;
    Pair* nodes;
    unsigned* status;
};
cudaError_t launch_poly_range(const float* f, size_t pitch, int H, int W, int R, int set_tile,
                              int sets_x, int n_sets, unsigned* mm, cudaStream_t s);
cudaError_t launch_poly_params(const PolyParamsArgs& a, cudaStream_t s);
cudaError_t launch_poly32(const FwdArgs& a, cudaStream_t s);   // a.cap_pairs = node entries
void poly_tile(int R, int cap_nodes, int* th, int* tw);

// Non-local means with a p-pixel patch (Sec. 6): the fused FP32 tile with
// the patch phase; one parameter set (fixed or image-wide T).
struct NlmPatch {
    int p;                  // patch pixels, u_1 = (0, 0) first
    int uy[9], ux[9];
    float sigma_r;
};
size_t nlm_smem_bytes(int R, int th, int tw, int n_cap);
void nlm_tile(int R, int n_cap, int* th, int* tw);
cudaError_t launch_nlm32(const FwdArgs& a, const NlmPatch& pt, int n_cap, cudaStream_t s);
// Box spatial filter with FP32 planes by exact integer running sums (any R
// up to 63): output rows of its tile (0 when none fits), the launch.
int box32_rows(int R, int set_tile);
cudaError_t launch_box32(const FwdArgs& a, cudaStream_t s);
// K3-sep (FP32 FIR in two passes through HBM, R > 24, one parameter set).
struct SepArgs {
    const float* f;
    size_t f_pitch;
    float* out;
    size_t out_pitch;
    int H, W, Wp, R;        // Wp: row stride of P (multiple of 128)
    float c0;
    const SetHdr* hdr;
    const Pair* pairs;
    const float* taps;      // device taps (guard mass)
    const float* h_taps;    // host taps (kernel parameter)
    float2* P;              // [nk][2][H][Wp]: pairs (f'c, f's), (c, s)
    float2* nd;             // [H][W]
    int nk;                 // terms per chunk
    unsigned long long* n_guarded;
    float* den_out;
    size_t den_pitch;
    unsigned* fix_list = nullptr;   // FP32 recheck list of the one set (null: off)
    unsigned* fix_count = nullptr;
    float fix_kappa = 0.f;
};
bool sep32_ok(int R);
int sep32_width(int W);
cudaError_t launch_sep32(const SepArgs& a, int n_terms_cap, cudaStream_t s);

// Output tile of the FP32 kernel for a given R (0 if unsupported).
void fwd32_tile(int R, int* th, int* tw);
size_t fwd32_smem(int R, int th, int tw);
bool fwd32t_ok(int R, int set_tile);   // the tall tile serves this launch
int fwd32t_rows(int set_tile);         // its output rows (128, or 64 for 64-row T-tiles)
cudaError_t launch_fwd32(const FwdArgs& a, cudaStream_t s);

// K5 (adjoint, FP32 planes, FIR): needs the forward's out and den images.
struct BwdArgs {
    const float* h_taps;    // host copy of the taps (null: shared-memory taps only)
    const float* f;
    const float* u;         // dL/d out
    float* grad;            // dL/d f
    size_t pitch;           // of f, u, grad
    const float* out;       // forward output (scratch)
    const float* den;       // forward denominator (scratch)
    size_t spitch;          // of out, den
    int H, W, R;
    const float* taps;
    const SetHdr* hdr;
    const Pair* pairs;
    int cap_pairs;
    int set_tile;
    int sets_x;
    float c0;
};
void bwd32_tile(int R, int* th, int* tw);

// K3-yvv (recursive spatial filter): first-order sections of the Young-van
// Vliet recursion's poles, as FP32 (p0 real pole, p1 = Pr + i Pi; causal
// output C0 u0 + Cr Re u1 - Ci Im u1, anti-causal output D0 v0 + Dr Re v1 -
// Di Im v1).
struct YvvCoef {
    float P0, Pr, Pi;
    float C0, Cr, Ci;
    float D0, Dr, Di;
};
// The same coefficients as (x, x) pairs for packed multiply-adds (nPi = -Pi ...).
struct YvvCoef2 {
    float2 P0, Pr, Pi, nPi;
    float2 C0, Cr, nCi;
    float2 D0, Dr, nDi;
};
struct YvvArgs {
    const float* f;
    size_t f_pitch;
    float* out;
    size_t out_pitch;
    int H, W;
    float c0;
    const SetHdr* hdr;
    const Pair* pairs;
    int G;                  // pass groups per launch (G * C = 32 term columns)
    int n_nd;               // (num, den) partials summed by the final kernel
    float4* P;              // [H][W][G * C] row-filtered planes (f'c, c, f's, s)
    float4* S;              // [H][ceil(W/8)][3][G * C] anti-causal row states
    float2* nd;             // [G][H][W] (num, den) partials
    const float* mass_y;    // [H]
    const float* mass_x;    // [W]
    unsigned long long* n_guarded;
    YvvCoef coef;
    YvvCoef2 coef2;
};
// Plan-time design (false when sigma < 0.5, outside the recursion's range);
// poles_c (may be null) receives p0, Re p1, Im p1, c0, Re c1, Im c1.
bool yvv_design(double sigma, YvvCoef* out, double* poles_c);
void yvv_line_mass(double sigma, int n, float* mass);
int yvv_terms_per_pass(int n_terms_cap);
cudaError_t launch_yvv(const YvvArgs& a, int C, int n_passes, cudaStream_t s);
cudaError_t launch_bwd32(const BwdArgs& a, cudaStream_t s);

// ---- batched path (bf_execute_batch) ----------------------------------------
struct RangeImg {
    const float* f;
    size_t pitch;
    int H, W, R, set_tile, sets_x;
    unsigned* Tbits;
};
int range_tile();
size_t range_smem_bytes(int R);
cudaError_t launch_local_range_batch(const RangeImg* imgs, const int4* items, int n_items,
                                     int max_R, bool with_min, int n_ctas, cudaStream_t s);
cudaError_t launch_params_batch(const ParamsArgs* imgs, const int* block_img, const int* block_set,
                                int n_blocks, cudaStream_t s);
cudaError_t launch_fwd32_persistent(int th, int tw, int max_R, const FwdArgs* imgs,
                                   const int4* items, int n_items, unsigned* head, int n_ctas,
                                   cudaStream_t s);
int fwd32_persistent_ctas_per_sm(int th, int tw, int max_R);
FwdArgs forward_args(bf_plan_s* p, const float* f, size_t fp, float* out, size_t op);
ParamsArgs plan_params_args(bf_plan_s* p);
void batch_forget(bf_plan_s* p);

// K3-tc (FP16 / BF16 planes, tcgen05): 128 x 32 output tiles, R <= max radius.
int fwd_tc_max_radius();
void fwd_tc_tile(int* th, int* tw);
cudaError_t launch_fwd_tc(const FwdArgs& a, bool bf16, long long spin_limit, unsigned* status,
                          cudaStream_t s);

}  // namespace bf
