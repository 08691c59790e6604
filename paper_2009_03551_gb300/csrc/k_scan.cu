// Exclusive prefix sums used to turn per-row / per-slot counts into offsets.
// Three launches: per-tile sums, a single-CTA scan of the tile sums, and the
// per-tile scan with the tile offset added.  out[n] receives the total; an
// initial value `init` is added to every output.
// The scan is deterministic (integer addition).
#include "rdm_internal.cuh"

namespace rdm {
namespace {

constexpr int kThreads = 512;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

template <class T>
__device__ T block_exclusive_scan(T v, T *sh, T *total) {
    // warp-shuffle scan then scan of the warp totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = (lane < (kThreads / 32)) ? sh[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kThreads / 32)) sh[lane] = w;
    }
    __syncthreads();
    T excl = x - v + (wid > 0 ? sh[wid - 1] : T(0));
    if (total) *total = sh[kThreads / 32 - 1];
    __syncthreads();
    return excl;
}

template <class In, class Out>
__global__ void tile_sums(const In *__restrict__ in, int n, Out *__restrict__ tile_sum) {
    __shared__ Out sh[32];
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    Out s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n) s += (Out)in[base + k];
    Out tot;
    block_exclusive_scan<Out>(s, sh, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

template <class Out>
__global__ void scan_tiles(Out *tile_sum, int ntiles, Out *total_out, Out init) {
    __shared__ Out sh[32];
    Out carry = init;
    for (int base = 0; base < ntiles; base += kThreads) {
        int i = base + threadIdx.x;
        Out v = i < ntiles ? tile_sum[i] : Out(0);
        Out tot;
        Out e = block_exclusive_scan<Out>(v, sh, &tot);
        if (i < ntiles) tile_sum[i] = e + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <class In, class Out>
__global__ void scan_apply(const In *in, int n, const Out *__restrict__ tile_sum, Out *out) {
    __shared__ Out sh[32];
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    Out v[kItems];
    Out s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = (base + k < n) ? (Out)in[base + k] : Out(0);
        s += v[k];
    }
    Out e = block_exclusive_scan<Out>(s, sh, nullptr) + tile_sum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n) out[base + k] = e;
        e += v[k];
    }
}

template <class In, class Out>
void scan_impl(const In *in, Out *out, int n, Out *tmp, cudaStream_t st, Out init) {
    int ntiles = (n + kTile - 1) / kTile;
    if (ntiles < 1) ntiles = 1;
    tile_sums<In, Out><<<ntiles, kThreads, 0, st>>>(in, n, tmp);
    RDM_LAUNCH_CHECK();
    scan_tiles<Out><<<1, kThreads, 0, st>>>(tmp, ntiles, out + n, init);
    RDM_LAUNCH_CHECK();
    if (n > 0) {
        scan_apply<In, Out><<<ntiles, kThreads, 0, st>>>(in, n, tmp, out);
        RDM_LAUNCH_CHECK();
    }
}

}  // namespace

size_t scan_tmp_elems(int n) { return (size_t)((n + kTile - 1) / kTile + 1); }

void scan_exclusive_i32(const int *in, int *out, int n, int *tmp, cudaStream_t st, int init) {
    scan_impl<int, int>(in, out, n, tmp, st, init);
}
void scan_exclusive_i64(const int *in, int64_t *out, int n, int64_t *tmp, cudaStream_t st) {
    scan_impl<int, int64_t>(in, out, n, tmp, st, int64_t(0));
}

}  // namespace rdm
