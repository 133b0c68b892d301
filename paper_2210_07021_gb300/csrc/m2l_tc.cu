// M2L (Lemma 3) on the 5th-generation tensor cores, for the mixed path.
//
// With the translation parameters of expand.cu (a = c r_S, b = c r_T,
// g = (1 + c^2) r_S r_T, phases ph1, ph2) the scaled local contribution of one
// pair is, for l = 1..p,
//     Y_l = (b ph2)^l ( -Q/l + [B1 w]_l ),   w_n = rho^n [B2 u]_n,   rho = g/(a b),
//     u_l' = (a ph1)^l' X_l',
// with the fixed integer matrices B2[n][l'] = C(l', n) and B1[l][n] = C(l-1, n-1).
// Both stages are dense products with a matrix shared by every pair, so a tile
// of 64 pairs (rows 2j / 2j+1 = real / imaginary parts of pair j) is two
// [128 x PK] x [PK x PK] GEMMs (PK = 16 or 32, zero-padded).  FP32 operands are
// split into three BF16 terms (hi, mid, lo) and the binomials into two or three;
// the split products run as tcgen05.mma kind::f16 with FP32 accumulation in
// tensor memory (≈ 2^-24 relative, the FP32 level).  The diagonal scalings,
// the splits and the constant term C' = C + 2Q log sin(theta/2) + 2 Re sum u_l
// are done by the CTA's threads; each tile's outputs are summed per target
// segment and added to the (FP32) local expansions with atomics.
//
// rho = 1/cos^2(theta/2) grows without bound as the two centres approach
// antipodes; pairs with rho^PK beyond 2^100 are appended to a leftover list and
// translated by the warp kernel (k_m2l_list), which uses a, b, g directly.
//
// Operands in shared memory are K-major without swizzle: 8-row x 16-byte core
// matrices, core matrix (r/8, k/8) at (r/8) SBO + (k/8) LBO with LBO = 128 B
// (along K) and SBO = (PK/8) 128 B (along M or N).  One CTA of 128 threads
// (4 warps; warp w reads tensor-memory lanes 32w..32w+31) loops over tiles.
// Every mbarrier wait is bounded; on time-out the kernel sets an error word,
// waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include "common.cuh"

#include <cuda_bf16.h>

namespace sfmm {

namespace {

constexpr int TILE = 64;                 // pairs per tile
constexpr int WAIT_LIMIT = 1 << 26;

struct __align__(16) XGeo32T {             // same layout as expand.cu's XGeo32
    float a, b, g, logk;
    float p1x, p1y, p2x, p2y;
    float ar, ai, br, bi;
    float rho;
    int big;
    float pad[2];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__host__ __device__ __forceinline__ uint32_t kmaj_off(int r, int k, uint32_t sbo)
{
    return (uint32_t)((r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;          // LBO: next core matrix along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;  // SBO: next core matrix along M / N
    d |= (uint64_t)1 << 46;                   // descriptor version
    return d;
}

__device__ __forceinline__ void split3(float v, __nv_bfloat16* h, __nv_bfloat16* m, __nv_bfloat16* l)
{
    *h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(*h);
    *m = __float2bfloat16_rn(r1);
    *l = __float2bfloat16_rn(r1 - __bfloat162float(*m));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity)
{
    uint32_t done = 0;
    for (int it = 0; it < WAIT_LIMIT && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return done != 0;
}

template <int PK> struct TcSmem {
    static constexpr int SB = PK <= 16 ? 2 : 3;       // binomial splits: C(16,8) < 2^16; C(32,16) < 2^30
    static constexpr uint32_t SBO_A = (PK / 8) * 128;
    static constexpr uint32_t ABYTES = 128 * PK * 2;  // one split of a [128 x PK] BF16 tile
    static constexpr uint32_t BBYTES = PK * PK * 2;   // one split of a [PK x PK] BF16 tile
    alignas(1024) unsigned char a[3][ABYTES];
    alignas(1024) unsigned char b2[SB][BBYTES];
    alignas(1024) unsigned char b1[SB][BBYTES];
    float out[TILE][2 * PK + 2];      // per pair: C, Q, then (Re, Im) Y_1..Y_PK
    int tgt[TILE];
    float rho[TILE];
    uint64_t mbar;
    uint32_t tmem;
    int abort_flag;
};

template <int PK>
__device__ __forceinline__ void issue_stage(TcSmem<PK>* S, const unsigned char (*bm)[TcSmem<PK>::BBYTES], uint32_t dcol)
{
    constexpr int SB = TcSmem<PK>::SB;
    // idesc: D f32, A and B bf16, both K-major, N = PK, M = 128
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(PK >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    int first = 1;
    for (int ia = 0; ia < 3; ++ia)
        for (int ib = 0; ib < SB; ++ib) {
            if (ia + ib > 2) continue;            // products below 2^-24 relative are dropped
            for (int kb = 0; kb < PK / 16; ++kb) {
                const uint64_t da = umma_desc(smem_u32(S->a[ia]) + kb * 256, TcSmem<PK>::SBO_A);
                const uint64_t db = umma_desc(smem_u32(bm[ib]) + kb * 256, TcSmem<PK>::SBO_A);
                const uint32_t acc = first ? 0u : 1u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             :: "r"(S->tmem + dcol), "l"(da), "l"(db), "r"(idesc), "r"(acc));
                first = 0;
            }
        }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&S->mbar)) : "memory");
}

template <int PK>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float* v)
{
    for (int cb = 0; cb < PK / 16; ++cb) {
        uint32_t r[16];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                       "=r"(r[15])
                     : "r"(taddr + cb * 16));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) v[cb * 16 + j] = __uint_as_float(r[j]);
    }
}

template <int PK>
__global__ void __launch_bounds__(128) k_m2l_tc(int64_t n_pairs, const uint64_t* __restrict__ ptgt,
                                                const uint32_t* __restrict__ psrc, const XGeo32T* __restrict__ geo,
                                                const float* __restrict__ mpole, float* __restrict__ local, int p,
                                                uint32_t* __restrict__ leftover, uint32_t* __restrict__ n_leftover,
                                                int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem<PK>* S = reinterpret_cast<TcSmem<PK>*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int SB = TcSmem<PK>::SB;
    constexpr uint32_t SBO = TcSmem<PK>::SBO_A;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int j = tid >> 1, part = tid & 1;

    // binomial operands (K-major, rows = output index): B2 op[n][k] = C(k+1, n+1), B1 op[i][k] = C(i, k),
    // zero outside p x p; each split into BF16 terms of the FP64 integer (exact for p <= 16)
    for (int e = tid; e < PK * PK; e += blockDim.x) {
        const int r = e / PK, k = e % PK;
        double c2 = 0.0, c1 = 0.0;
        if (k >= r) { c2 = 1.0; for (int t = 0; t < r + 1; ++t) c2 = c2 * (k + 1 - t) / (t + 1); }   // C(k+1, r+1)
        if (k <= r) { c1 = 1.0; for (int t = 0; t < k; ++t) c1 = c1 * (r - t) / (t + 1); }           // C(r, k)
        if (r >= p || k >= p) { c2 = 0.0; c1 = 0.0; }
        double rem2 = c2, rem1 = c1;
        for (int sp = 0; sp < SB; ++sp) {
            const __nv_bfloat16 h2 = __float2bfloat16_rn((float)rem2), h1 = __float2bfloat16_rn((float)rem1);
            *(__nv_bfloat16*)(S->b2[sp] + kmaj_off(r, k, SBO)) = h2;
            *(__nv_bfloat16*)(S->b1[sp] + kmaj_off(r, k, SBO)) = h1;
            rem2 -= (double)__bfloat162float(h2);
            rem1 -= (double)__bfloat162float(h1);
        }
    }
    if (tid == 0) {
        S->abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&S->mbar)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&S->tmem)), "r"((uint32_t)(PK <= 16 ? 32 : 64)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    uint32_t phase = 0;
    bool pending = false;           // an MMA batch was committed and not yet waited for
    const int64_t n_tiles = (n_pairs + TILE - 1) / TILE;

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t k = tile * TILE + j;
        const bool valid = k < n_pairs;
        // ---------------- phase 1: u = (a ph1)^l' X_l', split into the A tiles
        float Xr[PK], Xi[PK];
        float rho = 0.f, bx = 0.f, by = 0.f, Cc = 0.f, Qs = 0.f;
        bool big = false;
        int t_node = -1;
        if (valid) {
            const XGeo32T G = geo[k];
            const int s = (int)psrc[k];
            t_node = (int)ptgt[k];
            const float* e = mpole + (size_t)s * EXP_STRIDE;     // rows are 8-byte aligned: float2 loads
            const float2 cq = *reinterpret_cast<const float2*>(e);
            Qs = cq.y;
            big = G.big != 0;
            rho = G.rho;
            const float ar = G.ar, ai = G.ai;
            bx = G.br;
            by = G.bi;
            float zr = 1.f, zi = 0.f, csum = 0.f;
#pragma unroll
            for (int l = 0; l < PK; ++l) {
                const float nr = zr * ar - zi * ai, ni = zr * ai + zi * ar;
                zr = nr; zi = ni;
                float xr = 0.f, xi = 0.f;
                if (l < p) {
                    const float2 x2 = *reinterpret_cast<const float2*>(e + 2 + 2 * l);
                    xr = x2.x;
                    xi = x2.y;
                }
                Xr[l] = zr * xr - zi * xi;
                Xi[l] = zr * xi + zi * xr;
                csum += Xr[l];
            }
            Cc = cq.x + 2.f * cq.y * G.logk + 2.f * csum;
            if (big && part == 0) {
                const uint32_t slot = atomicAdd(n_leftover, 1u);
                leftover[slot] = (uint32_t)k;
            }
        }
        if (!valid || big) {
#pragma unroll
            for (int l = 0; l < PK; ++l) { Xr[l] = 0.f; Xi[l] = 0.f; }
            Cc = 0.f; Qs = 0.f; rho = 0.f;
        }
        // the MMAs of the previous tile have been waited for (or none were issued)
#pragma unroll
        for (int l = 0; l < PK; ++l) {
            __nv_bfloat16 h, m, lo;
            split3(part ? Xi[l] : Xr[l], &h, &m, &lo);
            const uint32_t off = kmaj_off(tid, l, SBO);
            *(__nv_bfloat16*)(S->a[0] + off) = h;
            *(__nv_bfloat16*)(S->a[1] + off) = m;
            *(__nv_bfloat16*)(S->a[2] + off) = lo;
        }
        if (part == 0) {
            S->tgt[j] = valid ? t_node : -1;
            S->rho[j] = rho;
            S->out[j][0] = Cc;
            S->out[j][1] = Qs;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---------------- stage 1 GEMM: D1 = A * B2^T
        if (tid == 0) issue_stage<PK>(S, S->b2, 0);
        pending = true;
        if (!mbar_wait(&S->mbar, phase)) { atomicExch(status, SFMM_ETIMEOUT); S->abort_flag = 1; }
        else pending = false;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (S->abort_flag) break;
        // ---------------- w_n = rho^n [B2 u]_n, split into the A tiles
        float v[PK];
        tmem_load_row<PK>(S->tmem + lane_base, v);
        {
            const float r = S->rho[j];
            float rp = 1.f;
#pragma unroll
            for (int n = 0; n < PK; ++n) {
                rp *= r;
                __nv_bfloat16 h, m, lo;
                split3(v[n] * rp, &h, &m, &lo);
                const uint32_t off = kmaj_off(tid, n, SBO);
                *(__nv_bfloat16*)(S->a[0] + off) = h;
                *(__nv_bfloat16*)(S->a[1] + off) = m;
                *(__nv_bfloat16*)(S->a[2] + off) = lo;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---------------- stage 2 GEMM: D2 = A * B1^T
        if (tid == 0) issue_stage<PK>(S, S->b1, PK);
        pending = true;
        if (!mbar_wait(&S->mbar, phase)) { atomicExch(status, SFMM_ETIMEOUT); S->abort_flag = 1; }
        else pending = false;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (S->abort_flag) break;
        tmem_load_row<PK>(S->tmem + lane_base + PK, v);
        // ---------------- Y_l = (b ph2)^l (-Q/l + o_l)
        {
            float zr = 1.f, zi = 0.f;
#pragma unroll
            for (int l = 0; l < PK; ++l) {
                const float mine = v[l];
                const float other = __shfl_xor_sync(FULL, mine, 1);
                const float nr = zr * bx - zi * by, ni = zr * by + zi * bx;
                zr = nr; zi = ni;
                const float orr = (part ? other : mine) - Qs / (float)(l + 1);
                const float oi = part ? mine : other;
                const float y = part ? (zr * oi + zi * orr) : (zr * orr - zi * oi);
                S->out[j][2 + 2 * l + part] = (valid && !big) ? y : 0.f;
            }
        }
        __syncthreads();
        // ---------------- per-target segment sums, atomically added to the locals
        for (int c = tid; c < 2 * p + 2; c += blockDim.x) {
            int cur = -1;
            float acc = 0.f;
            for (int jj = 0; jj < TILE; ++jj) {
                const int tn = S->tgt[jj];
                if (tn != cur) {
                    if (cur >= 0 && acc != 0.f) atomicAdd(local + (size_t)cur * EXP_STRIDE + c, acc);
                    cur = tn;
                    acc = 0.f;
                }
                if (tn >= 0) acc += S->out[jj][c];
            }
            if (cur >= 0 && acc != 0.f) atomicAdd(local + (size_t)cur * EXP_STRIDE + c, acc);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // an MMA batch may still be in flight after a time-out: wait for it (bounded) before freeing
    if (pending) mbar_wait(&S->mbar, phase ^ 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(S->tmem), "r"((uint32_t)(PK <= 16 ? 32 : 64)) : "memory");
}

}  // namespace

size_t m2l_tc_smem_bytes(int pk)
{
    return (pk <= 16 ? sizeof(TcSmem<16>) : sizeof(TcSmem<32>)) + 1024;
}

cudaError_t launch_m2l_tc(int64_t n_pairs, const uint64_t* ptgt, const uint32_t* psrc, const void* geo,
                          const void* mpole, void* local, int p, uint32_t* leftover, uint32_t* n_leftover,
                          int* status, cudaStream_t s)
{
    if (n_pairs == 0) return cudaSuccess;
    const int64_t n_tiles = (n_pairs + TILE - 1) / TILE;
    int64_t grid = n_tiles < 152 * 8 ? n_tiles : 152 * 8;
    const XGeo32T* G = static_cast<const XGeo32T*>(geo);
    const float* mp = static_cast<const float*>(mpole);
    float* lc = static_cast<float*>(local);
    cudaError_t e;
    if (p <= 16) {
        const size_t smem = m2l_tc_smem_bytes(16);
        if ((e = cudaFuncSetAttribute(k_m2l_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_m2l_tc<16><<<(unsigned)grid, 128, smem, s>>>(n_pairs, ptgt, psrc, G, mp, lc, p, leftover, n_leftover,
                                                       status); count_launch();
    } else {
        const size_t smem = m2l_tc_smem_bytes(32);
        if ((e = cudaFuncSetAttribute(k_m2l_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        k_m2l_tc<32><<<(unsigned)grid, 128, smem, s>>>(n_pairs, ptgt, psrc, G, mp, lc, p, leftover, n_leftover,
                                                       status); count_launch();
    }
    return cudaGetLastError();
}

}  // namespace sfmm
