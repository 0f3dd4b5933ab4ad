// Device-wide exclusive scan of int32 items (Sec. 4.2: the offsets of the replicated pairs, and of
// the span slots of the binning by rows), reduce-then-scan over 4096-item tiles:
//   1. reduce: every block sums its tile (striped, coalesced reads) into partials[block];
//   2. partials: one block scans the block sums in place and writes the total;
//   3. downsweep: every block reads its tile striped into shared memory, each thread scans its 8
//      consecutive items there (blocked order), the block adds its partial, and the exclusive
//      prefixes go back out striped: every global read and write is coalesced.
// The items come from a functor f(j) (an array, a gathered array, or a quantity computed from the
// binning's records), so a transform that feeds a scan costs no pass of its own, and an epilogue
// functor may consume each prefix in the downsweep.  With out NULL only the total is produced
// (steps 1 and 2).  In-place use (out aliasing the functor's input,
// position j read only for item j) is safe: a block reads its whole tile before it writes.
#pragma once

#include "xpr_internal.cuh"

namespace xpr {
namespace {  // every translation unit that scans has its own copy of these kernels
namespace scan_detail {

constexpr int kThreads = 512;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 4096 (scan_partials_bytes depends on it)
constexpr int kPad = kTile + kTile / 32;  // shared copy padded by one word per 32 (conflict-free blocked reads)

__device__ __forceinline__ int padded(int i) { return i + (i >> 5); }

// Exclusive scan of one int64 per thread over the block; *total receives the block's sum.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *smem_warp, int64_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int64_t w = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) smem_warp[lane] = w;
    }
    __syncthreads();
    const int64_t prefix = wid > 0 ? smem_warp[wid - 1] : 0;
    *total = smem_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return prefix + x - v;
}

template <class F>
__global__ void __launch_bounds__(kThreads) reduce_kernel(F f, int64_t n, int64_t *__restrict__ partials) {
    grid_dep_wait();
    __shared__ int64_t sw[32];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int64_t j = base + (int64_t)k * kThreads + threadIdx.x;
        if (j < n) s += f(j);
    }
    int64_t tot;
    block_exclusive_scan(s, sw, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) partials_kernel(int64_t *__restrict__ partials, int64_t nb,
                                                            int64_t *__restrict__ total_out) {
    grid_dep_wait();
    __shared__ int64_t sw[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kThreads) {
        const int64_t j = base + threadIdx.x;
        const int64_t v = j < nb ? partials[j] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan(v, sw, &tot);
        if (j < nb) partials[j] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <class F, class Post>
__global__ void __launch_bounds__(kThreads) downsweep_kernel(F f, int32_t *out, int64_t n,
                                                             const int64_t *__restrict__ partials,
                                                             const int64_t *__restrict__ total, Post post) {
    grid_dep_wait();
    __shared__ int32_t s_v[kPad];
    __shared__ int64_t sw[32];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {  // striped, coalesced reads
        const int i = k * kThreads + t;
        const int64_t j = base + i;
        s_v[padded(i)] = j < n ? f(j) : 0;
    }
    __syncthreads();
    int32_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {  // this thread's 8 consecutive items
        v[k] = s_v[padded(t * kItems + k)];
        s += v[k];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan(s, sw, &tot) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        s_v[padded(t * kItems + k)] = (int32_t)ex;
        const int64_t j = base + t * kItems + k;
        if (j < n) post(j, ex, v[k]);
        ex += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k) {  // striped, coalesced writes
        const int i = k * kThreads + t;
        const int64_t j = base + i;
        if (j < n) out[j] = s_v[padded(i)];
    }
    if (blockIdx.x == 0 && t == 0) {
        out[n] = (int32_t)*total;
        post.finish(n, *total);
    }
}

}  // namespace scan_detail

// No epilogue: the default of launch_scan's post.
struct ScanNoPost {
    __device__ __forceinline__ void operator()(int64_t, int64_t, int32_t) const {}
    __device__ __forceinline__ void finish(int64_t, int64_t) const {}
};

// out[j] = sum_{k<j} f(k), out[n] = total (out NULL: the total only); the total (int64) goes to
// total_out, or to scan_total_ptr(partials, n) when total_out is NULL.  partials: at least
// scan_partials_bytes(n) bytes.  post (with out only): post(j, out[j], f(j)) runs for every item
// once its prefix is known, and post.finish(n, total) once, in the same kernel (for n > 0).
template <class F, class Post = ScanNoPost>
int launch_scan(F f, int32_t *out, int64_t n, void *partials, int64_t *total_out, cudaStream_t st,
                Post post = Post()) {
    using namespace scan_detail;
    const int64_t nb = (n + kTile - 1) / kTile;
    int64_t *part = reinterpret_cast<int64_t *>(partials);
    int64_t *tot = total_out ? total_out : scan_total_ptr(partials, n);
    if (n == 0) {
        if (out) XPR_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
        XPR_CUDA_TRY(cudaMemsetAsync(tot, 0, sizeof(int64_t), st));
        return XPR_OK;
    }
    XPR_CUDA_TRY(launch_dependent(reduce_kernel<F>, dim3((unsigned)nb), dim3(kThreads), 0, st, f, n, part));
    XPR_LAUNCH_CHECK("scan reduce_kernel");
    XPR_CUDA_TRY(launch_dependent(partials_kernel, dim3(1), dim3(kThreads), 0, st, part, nb, tot));
    XPR_LAUNCH_CHECK("scan partials_kernel");
    if (out) {
        XPR_CUDA_TRY(launch_dependent(downsweep_kernel<F, Post>, dim3((unsigned)nb), dim3(kThreads), 0, st, f, out,
                                      n, (const int64_t *)part, (const int64_t *)tot, post));
        XPR_LAUNCH_CHECK("scan downsweep_kernel");
    }
    return XPR_OK;
}

}  // namespace
}  // namespace xpr
