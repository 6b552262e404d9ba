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
//    and column col (N index 8 t + col, columns in groups of 8) and K index
//    a sK + j it holds digit t - a of W[j][col] (zero outside 0..L-1).  The
//    MMA with K slice a reads a shifted window of one digit buffer D per
//    column group (rows 8 (e + L - 1) + col for digit e), so D is written
//    once per step.
//  * TMEM then holds, for operand row m and diagonal t,
//    O_t = sum_{a+b=t} sum_j X_a[m][j] W_b[j][col], and X W = sum_t 256^t O_t.
//    The epilogue folds the 2L-1 diagonals with Montgomery constants
//    c_t = 256^t R mod q (split at bit 31, signed mad.wide products) in one
//    128-bit sum, reduces once (REDC, R = 2^64),
//    combines the X row with the A row of the same r through a lane shuffle
//    (rows 2r, 2r+1 sit in adjacent TMEM lanes), and writes the digits of
//    W_{i+1} back into D for the next step.
//
// Layouts are the no-swizzle K-major canonical form: a core matrix is 8
// rows x 16 bytes stored contiguously; core matrices adjacent in K are 128
// bytes apart (the descriptor's leading byte offset) and core matrices
// adjacent in M/N are one full K extent apart (the stride byte offset).
//
// Overlap: with c > 8 the two column groups are independent recurrences;
// warps 0-3 and 4-7 each own one (digit buffer, accumulator, completion
// barrier, MMA issuer), so one group's MMAs run while the other group folds.
// With c <= 8 the MMAs of a step are issued as two sets (diagonals below and
// above an even split point) with two commits; warps 0-3 fold the first set
// while the tensor core computes the second, and warps 4-7 fold the second.
// Measured on plane quintics (s = 45) the overlap hides little: the CUDA-core
// fold, reduction and digit writes take about 1.7 times the MMA issue and
// wait, and the sum of the two is what a step costs.
//
// Requirements: s <= 64 (2s operand rows in one M = 128 tile), c <= 16,
// q odd in [3, 2^60]; 256 threads; every wait on an MMA completion barrier
// is bounded by a %globaltimer deadline.
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
// accumulator columns of one column group (8 columns per diagonal) and rows of its digit buffer
__host__ __device__ inline int tc_N(int L) { return ((2 * L - 1) * 8 + 15) & ~15; }
__host__ __device__ inline int tc_drows(int L) { return tc_N(L) + (L - 1) * 8; }
// digits of q's residues: balanced digits cover |x| < 2^(8L-1) - 2^(8L-9), so
// 8L >= bits(q) + 2 suffices
__host__ __device__ inline int tc_digits(uint64_t q) {
    int bits = 0;
    while (bits < 64 && (q >> bits)) bits++;
    return (bits + 2 + 7) / 8;
}
// Per-block state of the tensor-core path.
struct TcState {
    uint16_t *Aop;      // 128 x (L sK) f16 digits
    uint16_t *Dop;      // two digit buffers of tc_drows(L) x sK f16 (one per column group)
    uint64_t *xbuf;     // 128 x 8 partial residues (diagonal split)
    uint32_t tmem;      // accumulator base (lane 0, first column)
    uint32_t mbar[2];   // shared addresses of the two completion barriers
    uint32_t phase[2];  // parity of their next completion (kept by threads 0 and 128)
    int L, sK;
    const uint2 *ct;    // c_t = 256^t R mod q as (low 31 bits, rest), t < 2L-1
    uint2 *ct_odd;      // [2][16]: per warp group, -i c_t mod q (same split) for its current step i
    uint64_t da0, db0;  // descriptors of the A operand and of the first digit buffer
};

// Shared-memory bytes of the two operands for the largest L, and of
// the 128 x 8 partial residues exchanged between the warp groups.
__host__ __device__ inline size_t tc_operand_bytes(int s) {
    const int sK = tc_sK(s);
    return (size_t)128 * kTcMaxL * sK * 2 + (size_t)2 * tc_drows(kTcMaxL) * sK * 2 + (size_t)128 * 8 * 8;
}
// Carve the operands out of the dynamic shared memory at p (sized for smax).
__device__ inline void tc_carve(TcState &S, unsigned char *p, int smax) {
    const int sK = tc_sK(smax);
    S.Aop = reinterpret_cast<uint16_t *>(p);
    S.Dop = S.Aop + (size_t)128 * kTcMaxL * sK;
    S.xbuf = reinterpret_cast<uint64_t *>(S.Dop + (size_t)2 * tc_drows(kTcMaxL) * sK);
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



// Offset (in f16 elements) of element (row, k) of a K-major no-swizzle
// operand whose K extent is kext.
__device__ __forceinline__ int tc_off(int row, int k, int kext) {
    return ((row >> 3) * (kext >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// Balanced digits by bytes: with y = x + sum_{a<L} 128 256^a (below 256^L
// for x < 2^(8L-2)), byte a of y minus 128 is digit a.  The f16 of an integer
// b - 128 (0 <= b < 256) is (1024 + b) - 1152, exact in f16: the bits of
// 1024 + b are 0x6400 | b.
__device__ __forceinline__ uint64_t digit_bias(int L) { return 0x8080808080808080ull >> (8 * (8 - L)); }

__device__ __forceinline__ uint16_t digit_half(uint64_t y, int a) {
    const uint32_t h = 0x6400u | (uint32_t)((y >> (8 * a)) & 0xFFu);
    uint16_t out;
    asm("{\n\t.reg .f16 x, m;\n\tmov.b16 x, %1;\n\tmov.b16 m, 0x6480;\n\tsub.f16 x, x, m;\n\tmov.b16 %0, x;\n\t}"
        : "=h"(out)
        : "h"((uint16_t)h));
    return out;
}

// Write the L balanced digits of x < q into operand row `row`, K index a kstride + j.
__device__ __forceinline__ void put_digits(uint16_t *op, int row, int j, int kstride, int kext, int L, uint64_t x) {
    const uint64_t y = x + digit_bias(L);
    for (int a = 0; a < L; a++) op[tc_off(row, a * kstride + j, kext)] = digit_half(y, a);
}

// Constants of modulus q for L digits: ct[t] = 256^t R mod q split as
// (low 31 bits, the rest).
__device__ inline void tc_constants(const ModQ &Q, int L, uint2 *ct) {
    if (threadIdx.x == 0) {
        uint64_t pw = 1 % Q.q;
        for (int t = 0; t < 2 * L - 1; t++) {
            const uint64_t m = to_mont(pw, Q);
            ct[t] = make_uint2((uint32_t)m & 0x7FFFFFFFu, (uint32_t)(m >> 31));
            pw = mul_small(pw, 256, Q);
        }
    }
}

// Descriptors of the chunk's operands (the address field advances by bytes / 16).
__device__ inline void tc_descriptors(TcState &S) {
    S.da0 = umma_desc(smem_u32(S.Aop), 128, (uint32_t)(S.L * S.sK * 16));
    S.db0 = umma_desc(smem_u32(S.Dop), 128, (uint32_t)(S.sK * 16));
}

// MMAs of one set: every K slice (a, jj) of the step, N accumulator columns
// from TMEM column col0, B rows from row0 of the digit buffer whose
// descriptor is db (before the Toeplitz shift of 8 (L-1-a) rows).
__device__ inline void tc_issue(const TcState &S, uint64_t db, uint32_t col0, int row0, int N) {
    const uint32_t idesc = umma_idesc_f16(128, N);
    tc_fence_after();
    uint32_t acc = 0;
    for (int a = 0; a < S.L; a++) {
        const uint64_t da = S.da0 + (uint64_t)(a * S.sK);
        const uint64_t dbr = db + (uint64_t)(((S.L - 1 - a) * 8 + row0) >> 3) * (uint64_t)S.sK;
        for (int jj = 0; jj < S.sK / 16; jj++) {
            tc_mma(S.tmem + col0, da + (uint64_t)(16 * jj), dbr + (uint64_t)(16 * jj), idesc, acc);
            acc = 1;
        }
    }
}

__device__ __forceinline__ void named_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// Wait (thread 0 for barrier 0, thread 128 for barrier 1) and record a timeout.
__device__ __forceinline__ void tc_wait_set(TcState &S, int g, int *s_abort) {
    const bool ok = mbar_wait(S.mbar[g], S.phase[g]);
    if (ok) S.phase[g] ^= 1u;  // on a timeout the caller waits once more on the same phase
    else s_abort[g] = 1;
}

__device__ __forceinline__ void madws(int64_t &acc, int a, int b) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// Sum over the diagonals t in [t0, t1) of O_t c_t for the first cn (<= 8)
// columns at TMEM address tl (this thread's lane), with c_t = c1 2^31 + c0
// (c0 < 2^31, c1 < 2^29) as two signed 64-bit sums S0 = sum O_t c0,
// S1 = sum O_t c1: |O_t| <= L sK 2^14 <= 2^23, so each stays below 2^58.
__device__ __forceinline__ void tc_fold(uint32_t tl, int t0, int t1, int cn, const uint2 *cst, int64_t (&S0)[8],
                                        int64_t (&S1)[8]) {
    for (int tb = t0; tb < t1; tb += 4) {
        uint32_t v[4][8];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (tb + u < t1) tmem_ld8(tl + (uint32_t)((tb + u) * 8), v[u]);
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (tb + u < t1) {
                const uint2 ctt = cst[tb + u];
#pragma unroll
                for (int cc = 0; cc < 8; cc++) {
                    if (cc < cn) {
                        const int o = __float2int_rn(__uint_as_float(v[u][cc]));
                        madws(S0[cc], o, (int)ctt.x);
                        madws(S1[cc], o, (int)ctt.y);
                    }
                }
            }
        }
    }
}

// REDC of S0 + 2^31 S1 + q 2^28 (a 128-bit value in (0, q 2^29): the offset
// makes the signed sum positive, |S0 + 2^31 S1| < 2T 2^23 q), i.e. the
// residue (S0 + 2^31 S1) R^{-1} mod q.
__device__ __forceinline__ uint64_t tc_reduce(int64_t S0, int64_t S1, const ModQ &Q) {
    const uint64_t l1 = (uint64_t)S1 << 31;
    int64_t hi = S1 >> 33;
    const uint64_t l2 = l1 + (uint64_t)S0;
    hi += (S0 >> 63) + (l2 < l1 ? 1 : 0);
    const uint64_t off = Q.q << 28;
    const uint64_t l3 = l2 + off;
    hi += (int64_t)(Q.q >> 36) + (l3 < l2 ? 1 : 0);
    return redc(l3, (uint64_t)hi, Q);
}

// Digits of W[r][col] (col within its group) into a digit buffer: row 8 (a + L - 1) + col, K index r.
__device__ __forceinline__ void tc_put_w(uint16_t *D, int L, int sK, int col, int r, uint64_t x) {
    const uint64_t y = x + digit_bias(L);
    for (int a = 0; a < L; a++) D[tc_off((a + L - 1) * 8 + col, r, sK)] = digit_half(y, a);
}

// k steps of Algorithm 2 with the operand A already holding X = M(k-1) and
// A (fenced for the async proxy).  Input W in `in` (s x cs limb pairs,
// [j cs + col]); the result goes to `out`.  Returns 1 (result in `out`) for
// k >= 1, 0 for k = 0, and -1 if an MMA wait timed out (the block must stop).
// s_abort: two shared flags.
__device__ inline int horner_block_tc(TcState &S, int s, int c, int k, const uint2 *in, uint2 *out, const ModQ &Q,
                                      int *s_abort) {
    if (k <= 0) return 0;
    const int cs = pad4(c);
    const int L = S.L, sK = S.sK, T = 2 * L - 1;
    const int N = tc_N(L), drows = tc_drows(L);
    const bool colsplit = c > 8;  // block-uniform
    const uint32_t MASK30 = (1u << 30) - 1;
    if (threadIdx.x == 0 || threadIdx.x == 128) tc_descriptors(S);
    if (threadIdx.x < 2) s_abort[threadIdx.x] = 0;
    // digit buffers: zero, then the digits of W
    {
        const int words = (colsplit ? 2 : 1) * drows * sK / 2;
        uint32_t *d32 = reinterpret_cast<uint32_t *>(S.Dop);
        for (int e = threadIdx.x; e < words; e += blockDim.x) d32[e] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
            const int j = e / c, col = e - j * c;
            const uint2 w = in[j * cs + col];
            tc_put_w(S.Dop + (size_t)(col >> 3) * drows * sK, L, sK, col & 7, j, ((uint64_t)w.y << 30) | w.x);
        }
        fence_async_smem();
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, group = warp >> 2;
    const int m = quarter * 32 + lane;
    const int r = m >> 1;
    const bool odd = (m & 1) != 0;
    const int tmid = (L + 1) & ~1;  // even: folded pairs never straddle the split
    const int N1 = min(tmid * 8, N);
    const bool two_sets = N1 >= 16 && N - N1 >= 16;
    int colbase, cn, t0, t1;
    uint32_t tcol;
    if (colsplit) {
        colbase = 8 * group;
        cn = min(8, c - colbase);
        t0 = 0;
        t1 = T;
        tcol = 128u * group;
    } else {
        colbase = 0;
        cn = c;
        t0 = group ? tmid : 0;
        t1 = group ? T : min(tmid, T);
        tcol = 0;
    }
    uint16_t *Dg = S.Dop + (size_t)(colsplit ? group : 0) * drows * sK;
    const uint64_t dbg = S.db0 + (uint64_t)(colsplit ? group : 0) * (uint64_t)(drows >> 3) * (uint64_t)sK;
    const uint32_t tl = S.tmem + ((uint32_t)(quarter * 32) << 16) + tcol;
    const bool leader = (threadIdx.x & 127) == 0;
    uint2 *cto = S.ct_odd + 16 * group;
    for (int i = 0; i < k; i++) {
        if (quarter == 1 && lane < T) {  // this group's constants of the A rows (factor -i)
            const uint64_t ct = ((uint64_t)S.ct[lane].y << 31) | S.ct[lane].x;
            const uint64_t x = mul_small(ct, (uint64_t)i, Q);
            const uint64_t y = x ? Q.q - x : 0;
            cto[lane] = make_uint2((uint32_t)y & 0x7FFFFFFFu, (uint32_t)(y >> 31));
        }
        if (colsplit) {
            if (leader) {
                tc_issue(S, dbg, tcol, 0, N);
                tc_commit(S.mbar[group]);
                tc_wait_set(S, group, s_abort);
            }
        } else {
            if (threadIdx.x == 0) {
                if (two_sets) {
                    tc_issue(S, dbg, 0, 0, N1);
                    tc_commit(S.mbar[0]);
                    tc_issue(S, dbg, (uint32_t)N1, N1, N - N1);
                } else {
                    tc_issue(S, dbg, 0, 0, N);
                    tc_commit(S.mbar[0]);
                }
                tc_commit(S.mbar[1]);
            }
            if (leader) tc_wait_set(S, group, s_abort);
        }
        named_sync(1 + group);
        bool aborted = s_abort[group] != 0;  // group-uniform
        tc_fence_after();
        const uint2 *cst = odd ? cto : S.ct;
        int64_t S0[8], S1[8];
#pragma unroll
        for (int cc = 0; cc < 8; cc++) { S0[cc] = 0; S1[cc] = 0; }
        if (!aborted && cn > 0 && t0 < t1) tc_fold(tl, t0, t1, cn, cst, S0, S1);
        if (!colsplit) {
            if (group == 1) {
#pragma unroll
                for (int cc = 0; cc < 8; cc++) S.xbuf[cc * 128 + m] = tc_reduce(S0[cc], S1[cc], Q);
            }
            __syncthreads();
            aborted = s_abort[0] || s_abort[1];  // block-uniform
        }
        if (aborted) break;
        if (colsplit || group == 0) {
            uint64_t val[8];
#pragma unroll
            for (int cc = 0; cc < 8; cc++) {
                const uint64_t x = tc_reduce(S0[cc], S1[cc], Q);
                val[cc] = colsplit ? x : addmod(x, S.xbuf[cc * 128 + m], Q.q);
            }
            const bool last = (i + 1 == k);
#pragma unroll
            for (int cc = 0; cc < 8; cc++) {
                const uint64_t other = __shfl_xor_sync(0xffffffffu, val[cc], 1);
                const uint64_t w = addmod(val[cc], other, Q.q);
                const bool mine = odd ? (cc >= 4) : (cc < 4);
                if (mine && r < s && cc < cn) {
                    if (last) out[r * cs + colbase + cc] = make_uint2((uint32_t)w & MASK30, (uint32_t)(w >> 30));
                    else tc_put_w(Dg, L, sK, cc, r, w);
                }
            }
        }
        tc_fence_before();
        fence_async_smem();
        if (colsplit) named_sync(1 + group);
        else __syncthreads();
    }
    __syncthreads();
    return (s_abort[0] || s_abort[1]) ? -1 : 1;
}

// TMEM allocation by warp 0 (kTcTmemCols columns) and barrier set-up; every
// thread of the block must call it.
__device__ inline void tc_setup(uint32_t *s_tmem, uint64_t *s_mbar /* [2] */) {
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(s_mbar)), "r"(1u) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(s_mbar + 1)), "r"(1u) : "memory");
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
