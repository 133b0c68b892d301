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
// [128 x PK] x [PK x PK] GEMMs (PK = 16 or 32, zero-padded; the threads form
// only the first PL = p rounded up to 8 columns).  FP32 operands are
// split into three BF16 terms (hi, mid, lo) and the binomials into two or three;
// the split products run as tcgen05.mma kind::f16 with FP32 accumulation in
// tensor memory (≈ 2^-24 relative, the FP32 level).  The diagonal scalings,
// the splits and the constant term C' = C + 2Q log sin(theta/2) + 2 Re sum u_l
// are done by the CTA's threads; each tile's outputs, staged in the bytes of
// its A tiles once the MMAs are complete, are summed per target segment (each
// half of the tile by its own thread per coefficient) and added to the (FP32)
// local expansions with atomics.
//
// rho = 1/cos^2(theta/2) grows without bound as the two centres approach
// antipodes; pairs with rho^PK beyond 2^100 are appended to a leftover list and
// translated by the warp kernel (k_m2l_list), which uses a, b, g directly.
//
// Operands in shared memory are K-major without swizzle: 8-row x 16-byte core
// matrices, core matrix (r/8, k/8) at (r/8) SBO + (k/8) LBO with LBO = 128 B
// (along K) and SBO = (PK/8) 128 B (along M or N).  One CTA of 128 threads
// (4 warps; warp w reads tensor-memory lanes 32w..32w+31) loops over tiles; the
// grid holds as many CTAs as the SMs keep resident.  Each thread writes its
// row's eight-column groups of one BF16 term as single 16-byte stores.
// Every mbarrier wait is bounded; on time-out the kernel sets an error word,
// waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include "common.cuh"
#include "xgeo.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

namespace sfmm {

namespace {

constexpr int TILE = 64;                 // pairs per tile
constexpr int TC_CTAS = 5;               // CTAs per SM: registers capped for 5; 5 x 64 TMEM columns <= 512
constexpr int WAIT_LIMIT = 1 << 26;

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

// Bounded wait on an mbarrier phase.  With a limit below WAIT_LIMIT (the test
// hook of sfmm_options.wait_limit) the polls are non-blocking test_wait, so a
// small limit runs out before the tensor core can finish; otherwise try_wait,
// which may suspend the thread between polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int limit = WAIT_LIMIT)
{
    uint32_t done = 0;
    if (limit < WAIT_LIMIT) {
        for (int it = 0; it < limit && !done; ++it)
            asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                         : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
        return done != 0;
    }
    for (int it = 0; it < WAIT_LIMIT && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return done != 0;
}

// Binomial coefficients C(n, k), n, k <= 33 (all below 2^31), from Pascal's rule
// at compile time.
struct BinomTable {
    uint32_t c[34][34];
};
constexpr BinomTable make_binom()
{
    BinomTable b{};
    for (int n = 0; n < 34; ++n) {
        b.c[n][0] = 1u;
        for (int k = 1; k <= n; ++k) b.c[n][k] = b.c[n - 1][k - 1] + b.c[n - 1][k];
    }
    return b;
}
__constant__ BinomTable kBinom = make_binom();

// An integer below 2^31 as up to three BF16 terms (hi, mid, lo) whose sum is the
// integer to 24 bits (exactly when it has at most 24 significant bits): each
// term is the BF16 rounding of the remainder, taken in integer arithmetic.
__device__ __forceinline__ void split_int_bf16(uint32_t c, int n, __nv_bfloat16* t)
{
    int64_t rem = c;
    for (int i = 0; i < n; ++i) {
        const float f = (float)rem;                      // |rem| < 2^31: one rounding to 24 bits
        t[i] = __float2bfloat16_rn(f);
        rem -= (int64_t)__bfloat162float(t[i]);           // the term is an integer (|term| >= 1) or 0
    }
}

// PK: padded order of the GEMMs (16 or 32).  PL: the orders the threads form
// (a multiple of 8, p <= PL <= PK); columns PL..PK-1 of the A tiles are zero.
template <int PK> struct TcSmem {
    static constexpr int SB = PK <= 16 ? 2 : 3;       // binomial splits: C(16,8) < 2^16; C(32,16) < 2^30
    static constexpr uint32_t SBO_A = (PK / 8) * 128;
    static constexpr uint32_t ABYTES = 128 * PK * 2;  // one split of a [128 x PK] BF16 tile
    static constexpr uint32_t BBYTES = PK * PK * 2;   // one split of a [PK x PK] BF16 tile
    static constexpr int OSTR = 2 * PK + 2;           // per pair: C, Q, then (Re, Im) Y_1..Y_PK
    // The A tiles; once the stage-2 MMAs of a tile have completed the same
    // bytes hold the per-pair outputs for the segment sums.
    union {
        unsigned char a[3][ABYTES];
        float out[TILE][OSTR];
    };
    unsigned char b2[SB][BBYTES];
    unsigned char b1[SB][BBYTES];
    int tgt[TILE];
    uint64_t mbar;
    uint32_t tmem;
    uint32_t next;                                    // the CTA's next tile
    int abort_flag;
};
static_assert(sizeof(float[TILE][TcSmem<16>::OSTR]) <= 3 * TcSmem<16>::ABYTES, "outputs fit in the A tiles");
static_assert(sizeof(float[TILE][TcSmem<32>::OSTR]) <= 3 * TcSmem<32>::ABYTES, "outputs fit in the A tiles");

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v)
{
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

// Eight consecutive K entries of one row, split into three BF16 terms (hi, mid,
// lo: v = hi + mid + lo to about 2^-24 relative), one 16-byte store per term.
template <int PK>
__device__ __forceinline__ void split3_store8(TcSmem<PK>* S, uint32_t off, const float* v)
{
    uint32_t wh[4], wm[4], wl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float x0 = v[2 * i], x1 = v[2 * i + 1];
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float r0 = x0 - __low2float(h), r1 = x1 - __high2float(h);
        const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
        const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - __low2float(m), r1 - __high2float(m));
        wh[i] = bf2_bits(h);
        wm[i] = bf2_bits(m);
        wl[i] = bf2_bits(l);
    }
    *reinterpret_cast<uint4*>(S->a[0] + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4*>(S->a[1] + off) = make_uint4(wm[0], wm[1], wm[2], wm[3]);
    *reinterpret_cast<uint4*>(S->a[2] + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

// one row of an A tile: the PL formed values, then zeros up to PK
template <int PK, int PL>
__device__ __forceinline__ void store_row(TcSmem<PK>* S, int row, const float* v)
{
#pragma unroll
    for (int c = 0; c < PL / 8; ++c) split3_store8<PK>(S, kmaj_off(row, 8 * c, TcSmem<PK>::SBO_A), v + 8 * c);
#pragma unroll
    for (int c = PL / 8; c < PK / 8; ++c) {
        const uint32_t off = kmaj_off(row, 8 * c, TcSmem<PK>::SBO_A);
#pragma unroll
        for (int t = 0; t < 3; ++t) *reinterpret_cast<uint4*>(S->a[t] + off) = make_uint4(0u, 0u, 0u, 0u);
    }
}

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

// NC chunks of 16 accumulator columns of this thread's row.  All loads are
// issued before the one wait; the empty asm statements after it tie every
// register to the wait, so no use of a loaded value can be scheduled earlier.
template <int NC>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float* v)
{
    uint32_t r[16 * NC];
#pragma unroll
    for (int cb = 0; cb < NC; ++cb)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(r[16 * cb + 0]), "=r"(r[16 * cb + 1]), "=r"(r[16 * cb + 2]), "=r"(r[16 * cb + 3]),
                       "=r"(r[16 * cb + 4]), "=r"(r[16 * cb + 5]), "=r"(r[16 * cb + 6]), "=r"(r[16 * cb + 7]),
                       "=r"(r[16 * cb + 8]), "=r"(r[16 * cb + 9]), "=r"(r[16 * cb + 10]), "=r"(r[16 * cb + 11]),
                       "=r"(r[16 * cb + 12]), "=r"(r[16 * cb + 13]), "=r"(r[16 * cb + 14]), "=r"(r[16 * cb + 15])
                     : "r"(taddr + cb * 16));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16 * NC; ++j) {
        asm volatile("" : "+r"(r[j]));
        v[j] = __uint_as_float(r[j]);
    }
}

__device__ __forceinline__ void tc_sync()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <int PK, int PL>
__global__ void __launch_bounds__(128, TC_CTAS) k_m2l_tc(int64_t n_pairs, const uint64_t* __restrict__ ptgt,
                                                const uint32_t* __restrict__ psrc, const XGeo32* __restrict__ geo,
                                                const float* __restrict__ mpole, float* __restrict__ local, int p,
                                                uint32_t* __restrict__ leftover, uint32_t* __restrict__ n_leftover,
                                                uint32_t* __restrict__ tile_ctr, int* __restrict__ status,
                                                int wait_limit)
{
    static_assert(PL % 8 == 0 && PL <= PK, "PL: a multiple of 8 up to PK");
    constexpr int NC = (PL + 15) / 16;            // accumulator chunks of 16 columns read back
    constexpr uint32_t TCOLS = PK <= 16 ? 32 : 64;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem<PK>* S = reinterpret_cast<TcSmem<PK>*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    constexpr int SB = TcSmem<PK>::SB;
    constexpr uint32_t SBO = TcSmem<PK>::SBO_A;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int j = tid >> 1, part = tid & 1;

    // binomial operands (K-major, rows = output index): B2 op[n][k] = C(k+1, n+1), B1 op[i][k] = C(i, k),
    // zero outside p x p; each split into BF16 terms of the FP64 integer (exact for p <= 16)
    for (int e = tid; e < PK * PK; e += blockDim.x) {
        const int r = e / PK, k = e % PK;
        uint32_t c2 = kBinom.c[k + 1][r + 1], c1 = kBinom.c[r][k];   // C(k+1, r+1), C(r, k) (0 when k < r / k > r)
        if (r >= p || k >= p) { c2 = 0u; c1 = 0u; }
        __nv_bfloat16 t2[SB], t1[SB];
        split_int_bf16(c2, SB, t2);
        split_int_bf16(c1, SB, t1);
        for (int sp = 0; sp < SB; ++sp) {
            *(__nv_bfloat16*)(S->b2[sp] + kmaj_off(r, k, SBO)) = t2[sp];
            *(__nv_bfloat16*)(S->b1[sp] + kmaj_off(r, k, SBO)) = t1[sp];
        }
    }
    if (tid == 0) {
        S->abort_flag = 0;
        S->next = atomicAdd(tile_ctr, 1u);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&S->mbar)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&S->tmem)), "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    uint32_t phase = 0;
    bool pending = false;           // an MMA batch was committed and not yet waited for
    const int64_t n_tiles = (n_pairs + TILE - 1) / TILE;
    const int ncol = 2 * p + 2;

    for (;;) {
        const int64_t tile = S->next;             // tiles are taken from a global counter, one per CTA at a time
        if (tile >= n_tiles) break;
        const int64_t k = tile * TILE + j;
        const bool valid = k < n_pairs;
        // ---------------- phase 1: u = (a ph1)^l' X_l' (this thread's part: Re or Im), split into the A tiles
        float u[PL];
        float rho = 0.f, bx = 0.f, by = 0.f, Cc = 0.f, Qs = 0.f;
        bool big = false;
        int t_node = -1;
        if (valid) {
            const XGeo32 G = geo[k];
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
            for (int l = 0; l < PL; ++l) {
                const float nr = zr * ar - zi * ai, ni = zr * ai + zi * ar;
                zr = nr; zi = ni;
                float xr = 0.f, xi = 0.f;
                if (l < p) {
                    const float2 x2 = *reinterpret_cast<const float2*>(e + 2 + 2 * l);
                    xr = x2.x;
                    xi = x2.y;
                }
                const float re = zr * xr - zi * xi;
                csum += re;
                u[l] = part ? zr * xi + zi * xr : re;
            }
            Cc = cq.x + 2.f * cq.y * G.logk + 2.f * csum;
            if (big && part == 0) {
                const uint32_t slot = atomicAdd(n_leftover, 1u);
                leftover[slot] = (uint32_t)k;
            }
        }
        if (!valid || big) {
#pragma unroll
            for (int l = 0; l < PL; ++l) u[l] = 0.f;
            Cc = 0.f; Qs = 0.f; rho = 0.f;
        }
        // the MMAs of the previous tile have been waited for (or none were issued)
        store_row<PK, PL>(S, tid, u);
        if (part == 0) S->tgt[j] = valid ? t_node : -1;
        tc_sync();
        // ---------------- stage 1 GEMM: D1 = A * B2^T
        if (tid == 0) issue_stage<PK>(S, S->b2, 0);
        pending = true;
        if (!mbar_wait(&S->mbar, phase, wait_limit)) { atomicExch(status, SFMM_ETIMEOUT); S->abort_flag = 1; }
        else pending = false;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (S->abort_flag) break;
        // ---------------- w_n = rho^n [B2 u]_n, split into the A tiles
        float v[16 * NC];
        tmem_load_row<NC>(S->tmem + lane_base, v);
        {
            float rp = 1.f;
#pragma unroll
            for (int n = 0; n < PL; ++n) {
                rp *= rho;
                v[n] *= rp;
            }
        }
        store_row<PK, PL>(S, tid, v);
        tc_sync();
        // ---------------- stage 2 GEMM: D2 = A * B1^T
        if (tid == 0) issue_stage<PK>(S, S->b1, PK);
        pending = true;
        if (!mbar_wait(&S->mbar, phase, wait_limit)) { atomicExch(status, SFMM_ETIMEOUT); S->abort_flag = 1; }
        else pending = false;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (S->abort_flag) break;
        tmem_load_row<NC>(S->tmem + lane_base + PK, v);
        // ---------------- Y_l = (b ph2)^l (-Q/l + o_l), staged over the A tiles (their MMAs are complete)
        {
            float zr = 1.f, zi = 0.f;
#pragma unroll
            for (int l = 0; l < PL; ++l) {
                const float mine = v[l];
                const float other = __shfl_xor_sync(FULL, mine, 1);
                const float nr = zr * bx - zi * by, ni = zr * by + zi * bx;
                zr = nr; zi = ni;
                const float orr = (part ? other : mine) - Qs * (1.f / (float)(l + 1));
                const float oi = part ? mine : other;
                const float y = part ? (zr * oi + zi * orr) : (zr * orr - zi * oi);
                if (l < p) S->out[j][2 + 2 * l + part] = (valid && !big) ? y : 0.f;
            }
            if (part == 0) {
                S->out[j][0] = Cc;
                S->out[j][1] = Qs;
            }
        }
        __syncthreads();
        // ---------------- per-target segment sums over each half of the tile, atomically added to the locals
        for (int it = tid; it < 2 * ncol; it += blockDim.x) {
            const int half = it >= ncol ? 1 : 0;
            const int c = it - half * ncol;
            const int j0 = half * (TILE / 2);
            int cur = -1;
            float acc = 0.f;
#pragma unroll 4
            for (int jj = j0; jj < j0 + TILE / 2; ++jj) {
                const int tn = S->tgt[jj];
                const float x = S->out[jj][c];
                if (tn != cur) {
                    if (cur >= 0 && acc != 0.f) atomicAdd(local + (size_t)cur * EXP_STRIDE + c, acc);
                    cur = tn;
                    acc = 0.f;
                }
                acc += x;             // rows of absent pairs hold zeros
            }
            if (cur >= 0 && acc != 0.f) atomicAdd(local + (size_t)cur * EXP_STRIDE + c, acc);
        }
        if (tid == 0) S->next = atomicAdd(tile_ctr, 1u);     // every thread read this tile's index before
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // an MMA batch may still be in flight after a time-out: wait for it (with the full bound,
    // whatever the limit of the waits above) before freeing the tensor memory it writes
    if (pending) mbar_wait(&S->mbar, phase ^ 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(S->tmem), "r"(TCOLS) : "memory");
}

template <int PK, int PL>
cudaError_t launch_inst(int64_t n_pairs, const uint64_t* ptgt, const uint32_t* psrc, const XGeo32* geo,
                        const float* mpole, float* local, int p, uint32_t* leftover, uint32_t* n_leftover,
                        uint32_t* tile_ctr, int* status, int wait_limit, cudaStream_t s)
{
    const size_t smem = sizeof(TcSmem<PK>) + 128;
    cudaError_t e;
    int dev = 0, sms = 0;
    if ((e = cudaFuncSetAttribute(k_m2l_tc<PK, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
        (e = cudaFuncSetAttribute(k_m2l_tc<PK, PL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)) ||
        (e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return e;
    // TC_CTAS per SM (what __launch_bounds__ sizes the registers for); every CTA
    // takes tiles from the counter until none are left, so the work balances
    // whatever the residency (CTAs an SM cannot hold yet start when others exit)
    const int64_t n_tiles = (n_pairs + TILE - 1) / TILE;
    const int64_t cap = (int64_t)sms * TC_CTAS;
    const int64_t grid = n_tiles < cap ? n_tiles : cap;
    k_m2l_tc<PK, PL><<<(unsigned)grid, 128, smem, s>>>(n_pairs, ptgt, psrc, geo, mpole, local, p, leftover, n_leftover,
                                                        tile_ctr, status, wait_limit);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_m2l_tc(int64_t n_pairs, const uint64_t* ptgt, const uint32_t* psrc, const void* geo,
                          const void* mpole, void* local, int p, uint32_t* leftover, uint32_t* n_leftover,
                          uint32_t* tile_ctr, int* status, int wait_limit, cudaStream_t s)
{
    if (n_pairs == 0) return cudaSuccess;
    if (wait_limit <= 0 || wait_limit > WAIT_LIMIT) wait_limit = WAIT_LIMIT;
    const XGeo32* G = static_cast<const XGeo32*>(geo);
    const float* mp = static_cast<const float*>(mpole);
    float* lc = static_cast<float*>(local);
    if (p <= 8) return launch_inst<16, 8>(n_pairs, ptgt, psrc, G, mp, lc, p, leftover, n_leftover, tile_ctr, status, wait_limit, s);
    if (p <= 16) return launch_inst<16, 16>(n_pairs, ptgt, psrc, G, mp, lc, p, leftover, n_leftover, tile_ctr, status, wait_limit, s);
    if (p <= 24) return launch_inst<32, 24>(n_pairs, ptgt, psrc, G, mp, lc, p, leftover, n_leftover, tile_ctr, status, wait_limit, s);
    return launch_inst<32, 32>(n_pairs, ptgt, psrc, G, mp, lc, p, leftover, n_leftover, tile_ctr, status, wait_limit, s);
}

}  // namespace sfmm
