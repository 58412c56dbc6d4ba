// K2: order N, truncation M and the pair table of phi_eps, per set, on
// device (the arithmetic is in bf_params.cuh).  One block per set; no host
// synchronisation.
#include "bf_params.cuh"

namespace bf {
namespace {

using params::kMaxTail;
using params::params_body;
constexpr int kThreads = 128;

__global__ void __launch_bounds__(kThreads) k_params(ParamsArgs a)
{
    __shared__ double tail[params::kTail];
    __shared__ int nm[2];
    params_body(a, a.set0 + blockIdx.x, tail, nm);
}

// Batched: block b computes set block_set[b] of image block_img[b].
__global__ void __launch_bounds__(kThreads)
k_params_batch(const ParamsArgs* __restrict__ imgs, const int* __restrict__ block_img,
               const int* __restrict__ block_set)
{
    __shared__ double tail[params::kTail];
    __shared__ int nm[2];
    const ParamsArgs a = imgs[block_img[blockIdx.x]];
    params_body(a, block_set[blockIdx.x], tail, nm);
}

}  // namespace

cudaError_t launch_params(const ParamsArgs& a, cudaStream_t s, int n)
{
    if (a.n_cap > kMaxTail) return cudaErrorInvalidValue;
    k_params<<<n > 0 ? n : a.n_sets, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_params_batch(const ParamsArgs* imgs, const int* block_img,
                                const int* block_set, int n_blocks, cudaStream_t s)
{
    k_params_batch<<<n_blocks, kThreads, 0, s>>>(imgs, block_img, block_set);
    return cudaGetLastError();
}

}  // namespace bf
