// Device-wide exclusive scans and a stable LSD radix sort of (u64 key, u32 value).
//
// Scan: reduce-then-scan in three launches (per-tile sums, a single-CTA scan of
// the tile sums, per-tile scans with the tile offset added).
// Sort: 8-bit digits; per pass one histogram launch (per tile of 2048 keys),
// one scan of the digit-major histogram, and one scatter launch that ranks the
// keys of each tile stably with warp match-any and per-warp digit counters.
#include "common.cuh"

namespace sfmm {

namespace {

constexpr int SC_T = 256, SC_I = 8, SC_TILE = SC_T * SC_I;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// block-wide exclusive scan of one value per thread (256 threads); returns the
// exclusive prefix and writes the block total to *total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* s_warp, T* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_incl_scan(v, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (SC_T / 32) ? s_warp[lane] : T(0);
        T wi = warp_incl_scan(w, lane);
        if (lane < (SC_T / 32)) s_warp[lane] = wi - w;
        if (lane == (SC_T / 32) - 1) *total = wi;
    }
    __syncthreads();
    return inc - v + s_warp[warp];
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, T* __restrict__ bsum)
{
    __shared__ T s_warp[SC_T / 32];
    __shared__ T s_total;
    const int64_t base = (int64_t)blockIdx.x * SC_TILE;
    T acc = 0;
    for (int r = 0; r < SC_I; ++r) {
        int64_t e = base + (int64_t)r * SC_T + threadIdx.x;
        if (e < n) acc += in[e];
    }
    block_excl_scan(acc, s_warp, &s_total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s_total;
}

template <typename T>
__global__ void k_scan_top(T* __restrict__ bsum, int64_t nb, T* __restrict__ total)
{
    __shared__ T s_warp[SC_T / 32];
    __shared__ T s_total;
    T carry = 0;
    for (int64_t c = 0; c < nb; c += SC_T) {
        int64_t e = c + threadIdx.x;
        T v = e < nb ? bsum[e] : T(0);
        T ex = block_excl_scan(v, s_warp, &s_total);
        if (e < nb) bsum[e] = ex + carry;
        carry += s_total;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void k_scan_down(const T* __restrict__ in, T* __restrict__ out, int64_t n, const T* __restrict__ bsum)
{
    __shared__ T s_tile[SC_TILE];
    __shared__ T s_warp[SC_T / 32];
    __shared__ T s_total;
    const int64_t base = (int64_t)blockIdx.x * SC_TILE;
    for (int r = 0; r < SC_I; ++r) {
        int64_t e = base + (int64_t)r * SC_T + threadIdx.x;
        s_tile[r * SC_T + threadIdx.x] = e < n ? in[e] : T(0);
    }
    __syncthreads();
    T loc[SC_I];
    T acc = 0;
    for (int i = 0; i < SC_I; ++i) { loc[i] = acc; acc += s_tile[threadIdx.x * SC_I + i]; }
    T ex = block_excl_scan(acc, s_warp, &s_total) + bsum[blockIdx.x];
    __syncthreads();
    for (int i = 0; i < SC_I; ++i) s_tile[threadIdx.x * SC_I + i] = loc[i] + ex;
    __syncthreads();
    for (int r = 0; r < SC_I; ++r) {
        int64_t e = base + (int64_t)r * SC_T + threadIdx.x;
        if (e < n) out[e] = s_tile[r * SC_T + threadIdx.x];
    }
}

template <typename T>
cudaError_t exclusive_scan_t(const T* in, T* out, int64_t n, T* total, void* tmp, cudaStream_t s)
{
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(T), s);
        return cudaSuccess;
    }
    const int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    T* bsum = static_cast<T*>(tmp);
    k_scan_reduce<T><<<(unsigned)nb, SC_T, 0, s>>>(in, n, bsum); count_launch();
    k_scan_top<T><<<1, SC_T, 0, s>>>(bsum, nb, total); count_launch();
    k_scan_down<T><<<(unsigned)nb, SC_T, 0, s>>>(in, out, n, bsum); count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_T = 256, RS_I = 8, RS_TILE = RS_T * RS_I, RS_W = RS_T / 32;

__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
                          int64_t ntiles)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_I; ++r) {
        int64_t e = base + (int64_t)r * RS_T + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                             uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                             const uint32_t* __restrict__ offs, int64_t ntiles)
{
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[RS_W][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_I; ++r) {
        for (int k = tid; k < RS_W * 256; k += RS_T) (&wc[0][0])[k] = 0;
        __syncthreads();
        const int64_t e = tile0 + (int64_t)r * RS_T + tid;
        const bool valid = e < n;
        const uint64_t key = valid ? kin[e] : 0ull;
        const uint32_t val = valid ? vin[e] : 0u;
        const int d = valid ? (int)((key >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(FULL, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = base[tid];
            for (int w = 0; w < RS_W; ++w) { uint32_t c = wc[w][tid]; wc[w][tid] = acc; acc += c; }
            base[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t p = wc[warp][d] + (uint32_t)rank;
            kout[p] = key;
            vout[p] = val;
        }
        __syncthreads();
    }
}

}  // namespace

size_t scan_tmp_bytes(int64_t n)
{
    int64_t nb = (n + SC_TILE - 1) / SC_TILE + 1;
    return (size_t)nb * sizeof(int64_t) + 256;
}

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s)
{
    return exclusive_scan_t<int64_t>(in, out, n, total, tmp, s);
}

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* tmp, cudaStream_t s)
{
    return exclusive_scan_t<uint32_t>(in, out, n, total, tmp, s);
}

size_t radix_tmp_bytes(int64_t n)
{
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const int64_t nh = 256 * ntiles;
    // histogram + scanned histogram + scan scratch
    return (size_t)(2 * nh) * sizeof(uint32_t) + scan_tmp_bytes(nh) + 512;
}

cudaError_t radix_sort(uint64_t* k1, uint32_t* v1, uint64_t* k2, uint32_t* v2, int64_t n, int bits,
                       void* tmp, cudaStream_t s, bool* in_alt)
{
    *in_alt = false;
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const int64_t nh = 256 * ntiles;
    uint32_t* hist = static_cast<uint32_t*>(tmp);
    uint32_t* offs = hist + nh;
    void* stmp = reinterpret_cast<char*>(tmp) + (size_t)(2 * nh) * sizeof(uint32_t);
    stmp = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(stmp) + 255) & ~uintptr_t(255));
    uint64_t *ka = k1, *kb = k2;
    uint32_t *va = v1, *vb = v2;
    bool alt = false;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, RS_T, 0, s>>>(ka, n, shift, hist, ntiles); count_launch();
        cudaError_t e = exclusive_scan_u32(hist, offs, nh, nullptr, stmp, s);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<(unsigned)ntiles, RS_T, 0, s>>>(ka, va, kb, vb, n, shift, offs, ntiles); count_launch();
        std::swap(ka, kb);
        std::swap(va, vb);
        alt = !alt;
    }
    *in_alt = alt;
    return cudaGetLastError();
}

}  // namespace sfmm
