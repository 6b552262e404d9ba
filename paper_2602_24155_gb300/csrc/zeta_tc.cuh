// Limb-split modular GEMM steps on the 5th-generation tensor cores (tcgen05).
//
// One step of Algorithm 2 inside a chunk of k steps is
//   W_{i+1} = M(k-1-i) W_i = X W_i - i (A W_i)  mod q,   X = M(k-1) = R_{U-v,v},
// (Prop. 3.3: M(y) = y A + B is affine in the step index), a product of an
// s x s residue matrix with an s x c residue matrix.  It runs exactly on the
// tensor cores as an fp16 GEMM with fp32 accumulation:
//
//  * Residues x < q are written with L balanced base-256 digits,
//    x = sum_a d_a 256^a, d_a in [-128, 127]; such digits are exact in fp16,
//    a digit product is at most 2^14 in magnitude, and a sum of L * sK <= 512
//    of them stays within 2^23, so every fp32 partial sum is an exact integer.
//  * The A operand (128 rows, K = L * sK) holds the digits of X in the even
//    rows 2r and of A in the odd rows 2r + 1, digit a of column j at
//    K index a sK + j.
//  * The B operand is a Toeplitz stack of W's digits: for output diagonal t
//    and column col (N index t cp + col) and K index a sK + j it holds digit
//    t - a of W[j][col] (zero outside 0..L-1).  The MMA with K slice a reads
//    a shifted window of one digit buffer D (rows (e + L - 1) cp + col for
//    digit e), so D is written once per step.
//  * TMEM then holds, for operand row m and diagonal t,
//    O_t = sum_{a+b=t} sum_j X_a[m][j] W_b[j][col], and X W = sum_t 256^t O_t.
//    The epilogue folds the 2L-1 diagonals with Montgomery constants
//    c_t = 256^t R mod q in one 128-bit sum, reduces once (REDC, R = 2^64),
//    combines the X row with the A row of the same r through a lane shuffle
//    (rows 2r, 2r+1 sit in adjacent TMEM lanes), and writes the digits of
//    W_{i+1} back into D for the next step.
//
// Layouts are the no-swizzle K-major canonical form: a core matrix is 8
// rows x 16 bytes stored contiguously; core matrices adjacent in K are 128
// bytes apart (the descriptor's leading byte offset) and core matrices
// adjacent in M/N are one full K extent apart (the stride byte offset).
//
// Requirements: s <= 64 (2s operand rows in one M = 128 tile), c <= 16,
// q odd in [3, 2^60]; 256 threads; one MMA issuer (thread 0); every wait on
// the MMA completion barrier is bounded by a %globaltimer deadline.
#pragma once
#include <cuda_fp16.h>

namespace zeta {

constexpr int kTcMaxS = 64;
constexpr int kTcMaxC = 16;
constexpr int kTcMaxL = 8;
constexpr int kTcThreads = 256;
constexpr uint32_t kTcTmemCols = 256;
constexpr unsigned long long kTcWaitNs = 2000000000ull;  // 2 s per MMA wait

__host__ __device__ inline int tc_sK(int s) { return (s + 15) & ~15; }
__host__ __device__ inline int tc_cp(int c) { return c <= 8 ? 8 : 16; }
__host__ __device__ inline int tc_N(int L, int cp) { return ((2 * L - 1) * cp + 15) & ~15; }
__host__ __device__ inline int tc_drows(int L, int cp) { return tc_N(L, cp) + (L - 1) * cp; }
// digits of q's residues: balanced digits cover |x| < 2^(8L-1) - 2^(8L-9), so
// 8L >= bits(q) + 2 suffices
__host__ __device__ inline int tc_digits(uint64_t q) {
    int bits = 0;
    while (bits < 64 && (q >> bits)) bits++;
    return (bits + 2 + 7) / 8;
}
// Shared-memory bytes of the two operands for the largest L and cp.
__host__ __device__ inline size_t tc_operand_bytes(int s) {
    const int sK = tc_sK(s);
    return (size_t)128 * kTcMaxL * sK * 2 + (size_t)tc_drows(kTcMaxL, 16) * sK * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);  // descriptor version 1 (tcgen05), base offset 0, no swizzle
}

// kind::f16 instruction descriptor: A and B f16, D f32, both K-major, dense.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for completion of the barrier phase of the given parity, giving up
// after kTcWaitNs (returns false).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kTcWaitNs) return false;
    }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Per-block state of the tensor-core path.
struct TcState {
    uint16_t *Aop;      // 128 x (L sK) f16 digits
    uint16_t *Dop;      // drows x sK f16 digits
    uint32_t tmem;      // accumulator base (lane 0, first column)
    uint32_t mbar;      // shared address of the completion barrier
    uint32_t phase;     // parity of the next completion (thread 0)
    int L, sK, cp, N, drows;
    uint64_t bias;      // 2^23 sum_t 256^t mod q
    const uint2 *ct;    // c_t = 256^t R mod q as (low, high) 32-bit halves, t < 2L-1
};

// Offset (in f16 elements) of element (row, k) of a K-major no-swizzle
// operand whose K extent is kext.
__device__ __forceinline__ int tc_off(int row, int k, int kext) {
    return ((row >> 3) * (kext >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint16_t half_bits(int v) { return __half_as_ushort(__int2half_rn(v)); }

// Write the L balanced digits of x < q into operand row `row`, K index a kstride + j.
__device__ __forceinline__ void put_digits(uint16_t *op, int row, int j, int kstride, int kext, int L, uint64_t x) {
    for (int a = 0; a < L; a++) {
        int dg = (int)(x & 255u);
        x >>= 8;
        if (dg >= 128) { dg -= 256; x += 1; }
        op[tc_off(row, a * kstride + j, kext)] = half_bits(dg);
    }
}

// Constants of modulus q for L digits: ct[t] = 256^t R mod q, bias.
__device__ inline void tc_constants(const ModQ &Q, int L, uint2 *ct, uint64_t *bias) {
    if (threadIdx.x == 0) {
        uint64_t pw = 1 % Q.q, sum = 0;
        for (int t = 0; t < 2 * L - 1; t++) {
            const uint64_t m = to_mont(pw, Q);
            ct[t] = make_uint2((uint32_t)m, (uint32_t)(m >> 32));
            sum = addmod(sum, pw, Q.q);
            pw = mul_small(pw, 256, Q);
        }
        *bias = mul_small(sum, 1u << 23, Q);
    }
}

// Issue the MMAs of one step and wait for them (thread 0); returns false on timeout.
__device__ inline bool tc_step_mma(TcState &S) {
    const uint32_t a0 = smem_u32(S.Aop), d0 = smem_u32(S.Dop);
    const uint32_t sboA = (uint32_t)(S.L * S.sK * 16), sboD = (uint32_t)(S.sK * 16);
    const uint32_t idesc = umma_idesc_f16(128, S.N);
    tc_fence_after();
    uint32_t acc = 0;
    for (int a = 0; a < S.L; a++) {
        const uint32_t drow0 = (uint32_t)((S.L - 1 - a) * S.cp);  // multiple of 8
        for (int jj = 0; jj < S.sK / 16; jj++) {
            const uint32_t kA = (uint32_t)(a * S.sK + 16 * jj);
            const uint64_t da = umma_desc(a0 + (kA >> 3) * 128, 128, sboA);
            const uint64_t db = umma_desc(d0 + (drow0 >> 3) * sboD + (uint32_t)(2 * jj) * 128, 128, sboD);
            tc_mma(S.tmem, da, db, idesc, acc);
            acc = 1;
        }
    }
    tc_commit(S.mbar);
    const bool ok = mbar_wait(S.mbar, S.phase);
    if (ok) S.phase ^= 1u;  // on a timeout the caller waits once more on the same phase
    return ok;
}

// k steps of Algorithm 2 with the operand A already holding X = M(k-1) and
// A (fenced for the async proxy).  Input W in `in` (s x cs limb pairs,
// [j cs + col]); the result goes to `out`.  Returns 1 (result in `out`) for
// k >= 1, 0 for k = 0, and -1 if an MMA wait timed out (the block must stop).
__device__ inline int horner_block_tc(TcState &S, int s, int c, int k, const uint2 *in, uint2 *out, const ModQ &Q,
                                      int *s_abort) {
    if (k <= 0) return 0;
    const int cs = pad4(c);
    const int L = S.L, sK = S.sK, cp = S.cp;
    const uint32_t MASK30 = (1u << 30) - 1;
    // D: zero, then the digits of W
    {
        const int words = S.drows * sK / 2;
        uint32_t *d32 = reinterpret_cast<uint32_t *>(S.Dop);
        for (int e = threadIdx.x; e < words; e += blockDim.x) d32[e] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
            const int j = e / c, col = e - j * c;
            const uint2 w = in[j * cs + col];
            uint64_t x = ((uint64_t)w.y << 30) | w.x;
            for (int a = 0; a < L; a++) {
                int dg = (int)(x & 255u);
                x >>= 8;
                if (dg >= 128) { dg -= 256; x += 1; }
                S.Dop[tc_off((a + L - 1) * cp + col, j, sK)] = half_bits(dg);
            }
        }
        fence_async_smem();
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, colhalf = warp >> 2;
    const int m = quarter * 32 + lane;
    const int r = m >> 1;
    const bool odd = (m & 1) != 0;
    const bool active = colhalf * 8 < cp;  // warp-uniform
    const uint32_t tl = S.tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(colhalf * 8);
    for (int i = 0; i < k; i++) {
        if (threadIdx.x == 0) *s_abort = tc_step_mma(S) ? 0 : 1;
        __syncthreads();
        if (*s_abort) return -1;
        tc_fence_after();
        if (active) {
            uint64_t S0[8], S1[8];
#pragma unroll
            for (int cc = 0; cc < 8; cc++) { S0[cc] = 0; S1[cc] = 0; }
            for (int t = 0; t < 2 * L - 1; t++) {
                uint32_t v[8];
                tmem_ld8(tl + (uint32_t)(t * cp), v);
                tmem_wait_ld();
                const uint2 ctt = S.ct[t];
#pragma unroll
                for (int cc = 0; cc < 8; cc++) {
                    const uint32_t u = (uint32_t)(__float2int_rn(__uint_as_float(v[cc])) + (1 << 23));
                    madw(S0[cc], u, ctt.x);
                    madw(S1[cc], u, ctt.y);
                }
            }
            uint64_t val[8];
#pragma unroll
            for (int cc = 0; cc < 8; cc++) {
                uint64_t lo = S0[cc] + (S1[cc] << 32);
                const uint64_t hi = (S1[cc] >> 32) + (lo < S0[cc] ? 1ull : 0ull);
                uint64_t x = submod(redc(lo, hi, Q), S.bias, Q.q);
                if (odd) {
                    x = mul_small(x, (uint64_t)i, Q);
                    x = x ? Q.q - x : 0;
                }
                val[cc] = x;
            }
            const bool last = (i + 1 == k);
#pragma unroll
            for (int cc = 0; cc < 8; cc++) {
                const uint64_t other = __shfl_xor_sync(0xffffffffu, val[cc], 1);
                const uint64_t w = addmod(val[cc], other, Q.q);
                const int col = colhalf * 8 + cc;
                const bool mine = odd ? (cc >= 4) : (cc < 4);
                if (mine && r < s && col < c) {
                    if (last) {
                        out[r * cs + col] = make_uint2((uint32_t)w & MASK30, (uint32_t)(w >> 30));
                    } else {
                        uint64_t x = w;
                        for (int a = 0; a < L; a++) {
                            int dg = (int)(x & 255u);
                            x >>= 8;
                            if (dg >= 128) { dg -= 256; x += 1; }
                            S.Dop[tc_off((a + L - 1) * cp + col, r, sK)] = half_bits(dg);
                        }
                    }
                }
            }
        }
        tc_fence_before();
        fence_async_smem();
        __syncthreads();
    }
    return 1;
}

// TMEM allocation by warp 0 (kTcTmemCols columns) and barrier set-up; every
// thread of the block must call it.
__device__ inline void tc_setup(uint32_t *s_tmem, uint64_t *s_mbar) {
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(s_mbar)), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Release the accumulator columns (every thread calls; warp 0 frees).
__device__ inline void tc_teardown(uint32_t tmem) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

}  // namespace zeta
