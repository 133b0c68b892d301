// Device-wide exclusive scans and a stable LSD radix sort of (u64 key, u32 value).
//
// Scan: reduce-then-scan in three launches (per-tile sums, a single-CTA scan of
// the tile sums, per-tile scans with the tile offset added).
// Sort: 8-bit digits; per pass one histogram launch (per tile of 4096 keys),
// one scan of the digit-major histogram, and one scatter launch that ranks the
// keys of each tile stably (warp match-any, per-warp digit counters), reorders
// the tile by digit in shared memory and writes runs of equal digits.
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
// Tiles of RS_TILE = 4096 keys, 256 threads, 16 keys per thread.  Warp w owns
// keys [512 w, 512 w + 512) of its tile, loaded in 16 coalesced rounds of 32.
constexpr int RS_T = 256, RS_I = 16, RS_TILE = RS_T * RS_I, RS_W = RS_T / 32;
constexpr int RS_WC = 257;                        // per-warp digit counters (+1 slot for keys past n)
// the tile's keys, then its values, reordered through one 8-byte-per-key buffer,
// plus the digit of every reordered slot
constexpr size_t RS_SMEM = (size_t)RS_TILE * 9 + (size_t)RS_W * RS_WC * 4 + 3 * 256 * 4 + 64;

__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                 uint32_t* __restrict__ hist, int64_t ntiles)
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

// One tile: stable rank of every key among the tile's keys of its digit
// (warp-private counters advanced round by round; within a round the lanes of
// equal digit are found with eight ballots, one per digit bit), counts turned
// into per-warp offsets by a scan over (digit, warp), then the tile's keys and
// afterwards its values reordered by digit through one shared buffer and
// written out as runs per digit at the tile's global digit offsets (the
// scanned histogram).  Only the digits (packed four to a register) and the
// ranks stay in registers between the phases; keys and values are read again
// (from L2) when they are reordered, which keeps four CTAs on an SM.
__global__ void __launch_bounds__(RS_T, 4) k_rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                    uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                    int64_t n, int shift, const uint32_t* __restrict__ offs,
                                                    int64_t ntiles)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t* sk = reinterpret_cast<uint64_t*>(rs_smem);
    uint32_t* sv = reinterpret_cast<uint32_t*>(rs_smem);   // the same bytes, once the keys are out
    uint32_t* wc = reinterpret_cast<uint32_t*>(sk + RS_TILE);   // [RS_W][RS_WC]
    uint32_t* tbase = wc + RS_W * RS_WC;                  // tile-local start of each digit
    uint32_t* gbase = tbase + 256;                        // global start of this tile's keys of each digit
    uint32_t* s_warp = gbase + 256;                       // scan scratch
    uint8_t* sdig = reinterpret_cast<uint8_t*>(s_warp + 16);   // digit of each reordered slot
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    const int64_t w0 = tile0 + (int64_t)warp * (32 * RS_I);
    uint32_t dig[RS_I / 4];                               // digits, four to a register
    uint32_t loc[RS_I / 2];                               // slots (< 2^13), two to a register
#pragma unroll
    for (int r = 0; r < RS_I / 4; ++r) dig[r] = 0u;
#pragma unroll
    for (int r = 0; r < RS_I / 2; ++r) loc[r] = 0u;
#pragma unroll
    for (int r = 0; r < RS_I; ++r) {
        const int64_t e = w0 + r * 32 + lane;
        const uint32_t d = e < n ? (uint32_t)((kin[e] >> shift) & 255u) : 0u;
        dig[r >> 2] |= d << (8 * (r & 3));
    }
    for (int d = lane; d < RS_WC; d += 32) wc[warp * RS_WC + d] = 0;
    gbase[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RS_I; ++r) {
        const int64_t e = w0 + r * 32 + lane;
        const bool in = e < n;
        const int d = in ? (int)((dig[r >> 2] >> (8 * (r & 3))) & 255u) : 256;
        // lanes holding the same digit (keys past n: their own slot 256)
        unsigned peers = __ballot_sync(FULL, !in);
        peers = in ? ~peers : peers;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const unsigned m = __ballot_sync(FULL, (d >> b) & 1);
            peers &= ((d >> b) & 1) ? m : ~m;
        }
        const uint32_t before = wc[warp * RS_WC + d];
        __syncwarp();
        if ((peers & lt) == 0) wc[warp * RS_WC + d] = before + (uint32_t)__popc(peers);
        loc[r >> 1] |= (before + (uint32_t)__popc(peers & lt)) << (16 * (r & 1));
        __syncwarp();
    }
    __syncthreads();
    // thread tid = digit: per-warp exclusive offsets, then the tile's digit starts
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < RS_W; ++w) {
        const uint32_t c = wc[w * RS_WC + tid];
        wc[w * RS_WC + tid] = tot;
        tot += c;
    }
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t wv = lane < RS_W ? s_warp[lane] : 0u;
        uint32_t wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < RS_W) s_warp[lane] = wi - wv;
    }
    __syncthreads();
    tbase[tid] = inc - tot + s_warp[warp];
    __syncthreads();
    // keys to their places in the tile's digit order (read again, from L2)
#pragma unroll
    for (int r = 0; r < RS_I; ++r) {
        const int64_t e = w0 + r * 32 + lane;
        if (e < n) {
            const int d = (int)((dig[r >> 2] >> (8 * (r & 3))) & 255u);
            loc[r >> 1] += (tbase[d] + wc[warp * RS_WC + d]) << (16 * (r & 1));
            const uint32_t slot = (loc[r >> 1] >> (16 * (r & 1))) & 0xFFFFu;
            sk[slot] = kin[e];
            sdig[slot] = (uint8_t)d;
        }
    }
    __syncthreads();
    // runs of equal digits go to consecutive global positions: keys, then values
    const int cnt = (int)((n - tile0) < RS_TILE ? (n - tile0) : RS_TILE);
    for (int i = tid; i < cnt; i += RS_T) {
        const int d = sdig[i];
        kout[gbase[d] + (uint32_t)i - tbase[d]] = sk[i];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_I; ++r) {
        const int64_t e = w0 + r * 32 + lane;
        if (e < n) sv[(loc[r >> 1] >> (16 * (r & 1))) & 0xFFFFu] = vin[e];
    }
    __syncthreads();
    for (int i = tid; i < cnt; i += RS_T) {
        const int d = sdig[i];
        vout[gbase[d] + (uint32_t)i - tbase[d]] = sv[i];
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
    cudaError_t e = cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SMEM);
    if (e != cudaSuccess) return e;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, RS_T, 0, s>>>(ka, n, shift, hist, ntiles); count_launch();
        e = exclusive_scan_u32(hist, offs, nh, nullptr, stmp, s);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<(unsigned)ntiles, RS_T, RS_SMEM, s>>>(ka, va, kb, vb, n, shift, offs, ntiles); count_launch();
        std::swap(ka, kb);
        std::swap(va, vb);
        alt = !alt;
    }
    *in_alt = alt;
    return cudaGetLastError();
}

}  // namespace sfmm
