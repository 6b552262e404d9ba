// CUDA kernels of the controlled-reduction library (sm_103a).
//
// The hot path of arXiv 2602.24155: the linear recurrence of Sec. 3.2,
// W <- M(0) M(1) ... M(k-1) W mod p^M with M(y) = R_{x+yv,v} = y A + B
// (Prop. 3.3), evaluated as in Algorithm 2 (M <- (k-1)A + B; repeat
// { W <- M W; M <- M - A }), chunk after chunk as a reduction policy
// (Sec. 4) chooses directions v and chunk lengths k.
//
// Arithmetic: residues mod q = p^M < 2^60 in uint64.  A product of two
// residues is formed from 30-bit limbs with 32x32->64 multiply-adds
// (m = m1 2^30 + m0, w = w1 2^30 + w0), summed over blocks of 4 terms in
// 64-bit registers and then into 128-bit totals; one Montgomery reduction
// (Montgomery 1985, R = 2^64) per output folds the three limb sums.
//
// Step matrices are generated on the device from the section of the
// Jacobian map: for output monomial omega and input monomial mu,
//   R_{u,v}[omega, mu] = sum_i (u_i + omega_i) Sec[(i, omega - 1 + e_i), v + mu - 1]
// (the map g -> x^S sum_i (u_i g_i + x_i d_i g_i)/x_i of Prop. 3.3 written
// on monomials), so A[omega,mu] = sum_i v_i Sec[..] and
// B[omega,mu] = sum_i (x_i + omega_i) Sec[..].
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "zeta_internal.h"

namespace zeta {

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) {                                                         \
            err = std::string(#expr) + ": " + cudaGetErrorString(_e);                   \
            return ZETA_ERR_DEVICE;                                                      \
        }                                                                                \
    } while (0)

constexpr int kMaxS = 512;
constexpr int kMaxC = 32;

// ---------------------------------------------------------------------------
// Modular arithmetic on the device
// ---------------------------------------------------------------------------
struct ModQ {
    uint64_t q;
    uint64_t qneg_inv;  // -q^{-1} mod 2^64
    uint64_t r2;        // 2^128 mod q  (R^2, R = 2^64)
    uint64_t k30;       // 2^30 R mod q
};

__device__ __forceinline__ uint64_t mul_hi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// Montgomery reduction of T = hi 2^64 + lo < q 2^64: returns T 2^{-64} mod q.
__device__ __forceinline__ uint64_t redc(uint64_t lo, uint64_t hi, const ModQ &Q) {
    uint64_t m = lo * Q.qneg_inv;
    uint64_t ml = m * Q.q;
    uint64_t mh = mul_hi64(m, Q.q);
    uint64_t s = lo + ml;                 // low word is 0 by construction; carry matters
    uint64_t carry = (s < lo) ? 1ull : 0ull;
    uint64_t t = hi + mh + carry;
    return t >= Q.q ? t - Q.q : t;
}

// T mod q for T = hi 2^64 + lo < q 2^64.
__device__ __forceinline__ uint64_t reduce128(uint64_t lo, uint64_t hi, const ModQ &Q) {
    uint64_t y = redc(lo, hi, Q);
    return redc(y * Q.r2, mul_hi64(y, Q.r2), Q);
}

__device__ __forceinline__ uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}

__device__ __forceinline__ uint64_t submod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}

// a * small mod q, small < 2^32
__device__ __forceinline__ uint64_t mul_small(uint64_t a, uint64_t small, const ModQ &Q) {
    return reduce128(a * small, mul_hi64(a, small), Q);
}

__device__ __forceinline__ void add128(uint64_t &lo, uint64_t &hi, uint64_t x) {
    lo += x;
    hi += (lo < x) ? 1ull : 0ull;
}

// Limb layout of the recurrence.
//  W entries: 30-bit limbs (w0, w1) in a uint2 (q < 2^60), ordinary residues.
//  M entries: Montgomery form M R mod q in uint64, split on load into 20-bit
//             limbs m0, m1, m2.
// A limb product is below 2^50, so the six partial sums
//   S[t] = sum_j m_{t/2}(j) w_{t%2}(j)  (weights 2^{20 (t/2) + 30 (t%2)})
// stay below 2^59 for s <= 512 in plain uint64 registers.
// X = sum_j m_j w0_j and Y = sum_j m_j w1_j are each below s q 2^30 < q 2^64,
// so one Montgomery reduction (REDC, R = 2^64) applies to each:
//   (M W)_r = REDC(X) + REDC(REDC(Y) * (2^30 R mod q))  mod q.
__device__ __forceinline__ void madw(uint64_t &acc, uint32_t a, uint32_t b) {
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

__device__ __forceinline__ uint64_t fold_partials(const uint64_t S[6], const ModQ &Q) {
    uint64_t xl = S[0], xh = 0, yl = S[1], yh = 0;
    add128(xl, xh, S[2] << 20); xh += S[2] >> 44;
    add128(xl, xh, S[4] << 40); xh += S[4] >> 24;
    add128(yl, yh, S[3] << 20); yh += S[3] >> 44;
    add128(yl, yh, S[5] << 40); yh += S[5] >> 24;
    const uint64_t xr = redc(xl, xh, Q);   // X R^{-1}
    const uint64_t yr = redc(yl, yh, Q);   // Y R^{-1}
    const uint64_t c = redc(yr * Q.k30, mul_hi64(yr, Q.k30), Q);  // Y 2^30 R^{-1}
    return addmod(xr, c, Q.q);
}

// a R mod q (to Montgomery form)
__device__ __forceinline__ uint64_t to_mont(uint64_t a, const ModQ &Q) {
    return redc(a * Q.r2, mul_hi64(a, Q.r2), Q);
}

// ---------------------------------------------------------------------------
// One block-wide evaluation of k steps of Algorithm 2.
//  Ms, As: s x s uint64 in Montgomery form, entry (row r, col j) at
//          [j*s + r] (shared memory for small s, global scratch otherwise);
//          Ms holds M(k-1) R = ((k-1)A + B) R on entry and is consumed
//          (M <- M - A).
//  W, V  : s x cs limb pairs in shared memory, [j*cs + col], cs = c rounded
//          up to a multiple of 4 (the padding columns hold zeros and stay
//          zero); the input is in W; the output is in the buffer returned
//          (0 = W, 1 = V).
// Thread item = (row r, group of 4 consecutive columns); W is read 16 bytes
// (two columns) at a time.  The executor must stay at <= 96 registers per
// thread: above that a block of 160 threads takes more than a quarter of the
// register file and only three blocks fit an SM (4-way unrolling of the j loop
// reaches 100 with the executor's other state and runs the quintic batch 40 %
// slower).
// ---------------------------------------------------------------------------
__host__ __device__ inline int pad4(int c) { return (c + 3) & ~3; }

template <int CPT, bool L28 = false>
__device__ int horner_block(int s, int c, int k, uint64_t *Ms, const uint64_t *As, uint2 *W, uint2 *V,
                            const ModQ &Q) {
    static_assert(CPT == 4, "items are groups of four columns");
    const int cs = pad4(c);
    const int ngroups = cs / 4;
    const int items = s * ngroups;
    const uint32_t MASK20 = (1u << 20) - 1, MASK28 = (1u << 28) - 1, MASK30 = (1u << 30) - 1;
    // Few items (narrow W): split each item's j range between lanes l and
    // l + 16 of a warp and add the two partial sums with one shuffle round,
    // so that twice as many lanes work.  Block-uniform.
    const bool jsplit = 2 * items <= (int)blockDim.x;
    const int half = (int)((threadIdx.x >> 4) & 1u);
    int cur = 0;
    for (int step = 0; step < k; step++) {
        const uint2 *in = cur ? V : W;
        uint2 *out = cur ? W : V;
        for (int base = 0; base < items; base += jsplit ? items : (int)blockDim.x) {
            const int it = jsplit ? (int)((threadIdx.x >> 5) * 16 + (threadIdx.x & 15)) : base + (int)threadIdx.x;
            const bool valid = it < items;
            if (!jsplit && !valid) break;
            const int r = valid ? it % s : 0;
            const int c0 = valid ? (it / s) * 4 : 0;
            const int jb = (jsplit && half) ? s / 2 : 0;
            const int je = !valid ? jb : ((jsplit && !half) ? s / 2 : s);
            constexpr int NS = L28 ? 4 : 6;
            uint64_t S[4][NS];
#pragma unroll
            for (int cc = 0; cc < 4; cc++)
#pragma unroll
                for (int t = 0; t < NS; t++) S[cc][t] = 0;
            const int wstride = cs / 2;  // uint4 per W row
            const uint64_t *mp = Ms + (size_t)jb * s + r;
            const uint4 *wp = reinterpret_cast<const uint4 *>(in + c0) + (size_t)jb * wstride;
#pragma unroll 2
            for (int j = jb; j < je; j++) {
                const uint64_t m = *mp;
                mp += s;
                const uint4 wa = wp[0], wb = wp[1];  // columns c0, c0+1 | c0+2, c0+3
                wp += wstride;
                if (L28) {
                    // q < 2^56: 28-bit limbs of M (Montgomery form) and W, four products
                    const uint32_t m0 = (uint32_t)m & MASK28, m1 = (uint32_t)(m >> 28);
                    madw(S[0][0], m0, wa.x); madw(S[0][1], m0, wa.y); madw(S[1][0], m0, wa.z); madw(S[1][1], m0, wa.w);
                    madw(S[2][0], m0, wb.x); madw(S[2][1], m0, wb.y); madw(S[3][0], m0, wb.z); madw(S[3][1], m0, wb.w);
                    madw(S[0][2], m1, wa.x); madw(S[0][3], m1, wa.y); madw(S[1][2], m1, wa.z); madw(S[1][3], m1, wa.w);
                    madw(S[2][2], m1, wb.x); madw(S[2][3], m1, wb.y); madw(S[3][2], m1, wb.z); madw(S[3][3], m1, wb.w);
                } else {
                    const uint32_t m0 = (uint32_t)m & MASK20;
                    const uint32_t m1 = (uint32_t)(m >> 20) & MASK20;
                    const uint32_t m2 = (uint32_t)(m >> 40);
                    madw(S[0][0], m0, wa.x); madw(S[0][1], m0, wa.y);
                    madw(S[0][2], m1, wa.x); madw(S[0][3], m1, wa.y);
                    madw(S[0][4], m2, wa.x); madw(S[0][5], m2, wa.y);
                    madw(S[1][0], m0, wa.z); madw(S[1][1], m0, wa.w);
                    madw(S[1][2], m1, wa.z); madw(S[1][3], m1, wa.w);
                    madw(S[1][4], m2, wa.z); madw(S[1][5], m2, wa.w);
                    madw(S[2][0], m0, wb.x); madw(S[2][1], m0, wb.y);
                    madw(S[2][2], m1, wb.x); madw(S[2][3], m1, wb.y);
                    madw(S[2][4], m2, wb.x); madw(S[2][5], m2, wb.y);
                    madw(S[3][0], m0, wb.z); madw(S[3][1], m0, wb.w);
                    madw(S[3][2], m1, wb.z); madw(S[3][3], m1, wb.w);
                    madw(S[3][4], m2, wb.z); madw(S[3][5], m2, wb.w);
                }
            }
            if (jsplit) {
#pragma unroll
                for (int cc = 0; cc < 4; cc++)
#pragma unroll
                    for (int t = 0; t < NS; t++) S[cc][t] += __shfl_xor_sync(0xffffffffu, S[cc][t], 16);
                if (!valid || half) continue;
            }
            uint2 res[4];
#pragma unroll
            for (int cc = 0; cc < 4; cc++) {
                uint64_t v;
                if (L28) {
                    // X = S00 + (S01 + S10) 2^28 + S11 2^56 < s q^2 < q 2^64 (s <= 256)
                    uint64_t lo = S[cc][0], hi = 0;
                    add128(lo, hi, S[cc][1] << 28); hi += S[cc][1] >> 36;
                    add128(lo, hi, S[cc][2] << 28); hi += S[cc][2] >> 36;
                    add128(lo, hi, S[cc][3] << 56); hi += S[cc][3] >> 8;
                    v = redc(lo, hi, Q);
                    res[cc] = make_uint2((uint32_t)v & MASK28, (uint32_t)(v >> 28));
                } else {
                    v = fold_partials(S[cc], Q);
                    res[cc] = make_uint2((uint32_t)v & MASK30, (uint32_t)(v >> 30));
                }
            }
            uint4 *o = reinterpret_cast<uint4 *>(out + r * cs + c0);
            o[0] = make_uint4(res[0].x, res[0].y, res[1].x, res[1].y);
            o[1] = make_uint4(res[2].x, res[2].y, res[3].x, res[3].y);
        }
        __syncthreads();
        if (step + 1 < k) {
            for (int e = threadIdx.x; e < s * s; e += blockDim.x) Ms[e] = submod(Ms[e], As[e], Q.q);
            __syncthreads();
        }
        cur ^= 1;
    }
    return cur;
}

}  // namespace zeta
#include "zeta_tc.cuh"
namespace zeta {

// ---------------------------------------------------------------------------
// Device data of a batch
// ---------------------------------------------------------------------------
struct DInst {
    ModQ Q;
    uint32_t n, d, b, s, nv;
    uint32_t sec_rows, sec_cols, h_rows, kappa;
    uint32_t tab;          // table set index
    uint64_t sec_off;      // into sec pool
    uint32_t phase_off;    // into the phase offset pool: nphases + 1 entry offsets
    uint32_t nphases;
    uint32_t chain_base;   // global index of the instance's first chain
    uint32_t chunk_base;   // global index of the instance's first plan chunk
};

struct DTab {
    uint32_t nv, s, h_rows;
    uint32_t monoS_off;    // s*nv int32 exponents
    uint32_t secrow_off;   // nv*s int32 (row of Sec for (i, omega - 1 + e_i), -1 if invalid)
};

struct DChain {
    int32_t U[kMaxVars];
    uint32_t term_begin, term_end;
};

struct DEntry {
    int32_t U[kMaxVars];
    uint32_t chunk_begin, chunk_end;  // instance-relative
    int32_t arrival, start_chain, dest;
    uint32_t flags, live;
};

struct DChunk {
    int8_t v[kMaxVars];
    int32_t k;
};

__constant__ int32_t c_binom[64][9];  // C(a, b) for a < 64, b <= 8

__device__ __forceinline__ int dev_rank(const int *ex, int nv, int deg) {
    int idx = 0, rem = deg;
    for (int i = 0; i < nv - 1; i++) {
        int k = nv - i - 1;
        int top = rem - ex[i] - 1;
        if (top >= 0) idx += c_binom[top + k][k];
        rem -= ex[i];
    }
    return idx;
}

// Matrices M and A go to shared memory when both fit in this budget.
constexpr size_t kMatSmemBudget = 96 * 1024;
__host__ __device__ inline bool mats_in_smem(int s) { return (size_t)2 * s * s * sizeof(uint64_t) <= kMatSmemBudget; }

// Threads per block: one per (row, group of 4 columns) item, rounded to warps, 64..512.
inline int launch_threads(int s, int c) {
    int items = s * (pad4(c) / 4);
    int t = ((items + 31) / 32) * 32;
    return std::max(64, std::min(512, t));
}

// Shared-memory layout of the chain kernel (bytes): [M A] (if small), W, V,
// H partial, column map, colidx.
__host__ __device__ inline size_t chain_smem(int s, int c, int h_rows) {
    size_t bytes = 0;
    if (mats_in_smem(s)) bytes += (size_t)2 * s * s * sizeof(uint64_t);
    bytes += (size_t)2 * s * pad4(c) * sizeof(uint2);
    bytes += (size_t)h_rows * c * sizeof(uint64_t);
    bytes += (size_t)(c + s) * sizeof(int) + 64;
    return bytes;
}

// Persistent plan executor.  Each block takes instances from a queue
// (largest work first) and runs the instance's plan: phase after phase,
// entry after entry: form W from the arrival block and/or the start terms,
// play the entry's chunks (Algorithm 2 per chunk with matrices generated from
// the section), then store or add the result into the destination block of
// the next phase, or accumulate x^U g / x^S into H at pole order n.  One
// block owns an instance, so merges need no atomics.
template <int CPT, bool MSMEM, bool TC>
__global__ void __launch_bounds__(TC ? kTcThreads : 512) __maxnreg__(TC ? 255 : 96) k_execute(
    const DInst *__restrict__ insts, const DTab *__restrict__ tabs, const int32_t *__restrict__ tabpool,
    const uint64_t *__restrict__ secpool, const DChain *__restrict__ chains, const Term *__restrict__ terms,
    const uint32_t *__restrict__ phase_pool, const DEntry *__restrict__ entries, const DChunk *__restrict__ chunks,
    const uint32_t *__restrict__ order, uint32_t ninst, uint32_t *__restrict__ queue,
    uint64_t *__restrict__ scratch, size_t scratch_stride, uint64_t *__restrict__ blocks, size_t blocks_stride,
    uint64_t *__restrict__ Hout, size_t h_stride, unsigned long long *__restrict__ counters,
    unsigned long long *__restrict__ stamps) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int sU[kMaxVars], sv[kMaxVars], s_nlive;
    __shared__ uint32_t s_item;
    __shared__ uint32_t s_tmem;
    // Per-instance latency stamps are written by the cluster executor only: in this kernel any store added to
    // the instance loop, even one word per instance, measured 1.84x slower launches (same registers, no spills).
    (void)stamps;
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ uint2 s_ct[2 * kTcMaxL], s_ct_odd[2 * 16];
    __shared__ int s_abort[2];
    unsigned long long my_chunks = 0, my_steps = 0;
    TcState S;
    if (TC) {
        tc_setup(&s_tmem, s_mbar);
        S.tmem = s_tmem;
        S.mbar[0] = smem_u32(&s_mbar[0]);
        S.mbar[1] = smem_u32(&s_mbar[1]);
        S.phase[0] = S.phase[1] = 0;
        S.ct = s_ct;
        S.ct_odd = s_ct_odd;
    }
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t itx = s_item;
        __syncthreads();
        if (itx >= ninst) break;
        const uint32_t inst = order[itx];
        const DInst I = insts[inst];
        const DTab T = tabs[I.tab];
        const int s = (int)I.s, b = (int)I.b, nv = (int)I.nv, n = (int)I.n, d = (int)I.d;
        const int32_t *monoS = tabpool + T.monoS_off;
        const int32_t *secrow = tabpool + T.secrow_off;
        const uint64_t *Sec = secpool + I.sec_off;
        const uint32_t *ph = phase_pool + I.phase_off;
        unsigned char *ptr = smem_raw;
        uint64_t *Ms = nullptr, *As = nullptr;
        if (TC) {
            // operands sized for the largest s of the batch (scratch_stride)
            tc_carve(S, ptr, (int)scratch_stride);
            ptr += tc_operand_bytes((int)scratch_stride);
            S.sK = tc_sK(s);
            S.L = tc_digits(I.Q.q);
            tc_constants(I.Q, S.L, s_ct);
            uint32_t *a32 = reinterpret_cast<uint32_t *>(S.Aop);
            for (int e = threadIdx.x; e < 128 * S.L * S.sK / 2; e += blockDim.x) a32[e] = 0;
            __syncthreads();
        } else if (MSMEM) {
            Ms = (uint64_t *)ptr;
            As = Ms + (size_t)s * s;
            ptr += (size_t)2 * s * s * sizeof(uint64_t);
        } else {
            Ms = scratch + (size_t)blockIdx.x * scratch_stride;
            As = Ms + (size_t)s * s;
        }
        uint2 *W = (uint2 *)ptr;
        uint2 *V = W + (size_t)s * pad4(b);
        uint64_t *Hs = (uint64_t *)(V + (size_t)s * pad4(b));
        int *colmap = (int *)(Hs + (size_t)I.h_rows * b);
        int *colidx = colmap + b;
        uint64_t *bufA = blocks + (size_t)blockIdx.x * blocks_stride;
        uint64_t *bufB = bufA + blocks_stride / 2;
        // W limbs: 28 bits when q < 2^56 on the CUDA-core path (four products per entry), else 30 bits
        const bool l28 = !TC && I.Q.q < (1ull << 56) && s <= 256;
        const int lb = l28 ? 28 : 30;
        const uint32_t LMASK = (1u << lb) - 1u;
        for (int e = threadIdx.x; e < (int)I.h_rows * b; e += blockDim.x) Hs[e] = 0;
        for (uint32_t phase = 0; phase < I.nphases; phase++) {
            uint64_t *cur = (phase & 1) ? bufB : bufA;
            uint64_t *nxt = (phase & 1) ? bufA : bufB;
            for (uint32_t ei = ph[phase]; ei < ph[phase + 1]; ei++) {
                const DEntry E = entries[ei];
                if (threadIdx.x == 0) {
                    int nl = 0;
                    for (int col = 0; col < b; col++)
                        if (E.live >> col & 1u) colmap[nl++] = col;
                    s_nlive = nl;
                    for (int t = 0; t < nv; t++) sU[t] = E.U[t];
                }
                __syncthreads();
                const int c = s_nlive;
                const int cs = pad4(c);
                // W = arrival block (live columns) or 0; padding columns 0
                for (int e = threadIdx.x; e < s * cs; e += blockDim.x) {
                    const int j = e / cs, lc = e - j * cs;
                    uint64_t val = 0;
                    if (E.arrival >= 0 && lc < c) val = cur[(size_t)E.arrival * s * b + (size_t)j * b + colmap[lc]];
                    W[e] = make_uint2((uint32_t)val & LMASK, (uint32_t)(val >> lb));
                }
                __syncthreads();
                if (E.start_chain >= 0) {
                    // (row, column) is unique within a chain: the terms are added in parallel
                    const DChain C = chains[I.chain_base + E.start_chain];
                    for (uint32_t t = C.term_begin + threadIdx.x; t < C.term_end; t += blockDim.x) {
                        const Term tm = terms[t];
                        int lc = 0;
                        while (colmap[lc] != (int)tm.col) lc++;
                        const int e = (int)tm.row * cs + lc;
                        const uint64_t old = ((uint64_t)W[e].y << lb) | W[e].x;
                        const uint64_t nw = addmod(old, tm.coeff, I.Q.q);
                        W[e] = make_uint2((uint32_t)nw & LMASK, (uint32_t)(nw >> lb));
                    }
                }
                __syncthreads();
                int cur_buf = 0;  // 0: data in W, 1: data in V
                for (uint32_t ci = E.chunk_begin; ci < E.chunk_end; ci++) {
                    const DChunk CH = chunks[I.chunk_base + ci];
                    const int k = CH.k;
                    if (threadIdx.x < nv) sv[threadIdx.x] = CH.v[threadIdx.x];
                    __syncthreads();
                    // column index of v + mu - 1 in Homog_kappa (or -1)
                    for (int j = threadIdx.x; j < s; j += blockDim.x) {
                        int g[kMaxVars];
                        bool ok = true;
                        for (int t = 0; t < nv; t++) {
                            g[t] = sv[t] + monoS[j * nv + t] - 1;
                            if (g[t] < 0) ok = false;
                        }
                        colidx[j] = ok ? dev_rank(g, nv, (int)I.kappa) : -1;
                    }
                    __syncthreads();
                    // A R and M(k-1) R = R_{U-v,v} R from the section (held as Sec R mod q):
                    //   A[r,j] = sum_i v_i Sec[..],  M(k-1)[r,j] = sum_i (U_i - v_i + omega_i) Sec[..]
                    int res;
                    if (TC) {
                        // plain residues (one REDC removes R), as digits of the GEMM operand
                        const int kext = S.L * S.sK;
                        for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
                            const int r = e % s, j = e / s;
                            const int col = colidx[j];
                            uint64_t aL = 0, mL = 0, mH = 0;
                            if (col >= 0) {
                                for (int i = 0; i < nv; i++) {
                                    const int row = secrow[i * s + r];
                                    if (row < 0) continue;
                                    const uint64_t val = __ldg(&Sec[(size_t)row * I.sec_cols + col]);
                                    aL += val * (uint64_t)sv[i];
                                    const uint64_t wm = (uint64_t)(sU[i] - sv[i] + monoS[r * nv + i]);
                                    add128(mL, mH, val * wm);
                                    mH += mul_hi64(val, wm);
                                }
                            }
                            put_digits(S.Aop, 2 * r, j, S.sK, kext, S.L, redc(mL, mH, I.Q));
                            put_digits(S.Aop, 2 * r + 1, j, S.sK, kext, S.L, redc(aL, 0, I.Q));
                        }
                        fence_async_smem();
                        __syncthreads();
                        res = cur_buf == 0 ? horner_block_tc(S, s, c, k, W, V, I.Q, s_abort)
                                           : horner_block_tc(S, s, c, k, V, W, I.Q, s_abort);
                        if (res < 0) goto aborted;
                    } else {
                        for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
                            const int r = e % s, j = e / s;
                            const int col = colidx[j];
                            uint64_t aL = 0, mL = 0, mH = 0;
                            if (col >= 0) {
                                for (int i = 0; i < nv; i++) {
                                    const int row = secrow[i * s + r];
                                    if (row < 0) continue;
                                    const uint64_t val = __ldg(&Sec[(size_t)row * I.sec_cols + col]);
                                    aL += val * (uint64_t)sv[i];                       // < d q < 2^63
                                    const uint64_t wm = (uint64_t)(sU[i] - sv[i] + monoS[r * nv + i]);
                                    add128(mL, mH, val * wm);
                                    mH += mul_hi64(val, wm);
                                }
                            }
                            while (aL >= I.Q.q) aL -= I.Q.q;
                            As[(size_t)j * s + r] = aL;
                            Ms[(size_t)j * s + r] = reduce128(mL, mH, I.Q);
                        }
                        __syncthreads();
                        if (l28) res = cur_buf == 0 ? horner_block<CPT, true>(s, c, k, Ms, As, W, V, I.Q)
                                                    : horner_block<CPT, true>(s, c, k, Ms, As, V, W, I.Q);
                        else res = cur_buf == 0 ? horner_block<CPT, false>(s, c, k, Ms, As, W, V, I.Q)
                                                : horner_block<CPT, false>(s, c, k, Ms, As, V, W, I.Q);
                    }
                    cur_buf ^= res;
                    if (threadIdx.x == 0) {
                        for (int t = 0; t < nv; t++) sU[t] -= k * sv[t];
                        my_chunks++;
                        my_steps += k;
                    }
                    __syncthreads();
                }
                const uint2 *R = cur_buf ? V : W;
                if (E.dest < 0) {
                    // pole order n: accumulate x^U g / x^S into H
                    const int hdeg = d * n - n - 1;
                    for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
                        const int j = e / c, lc = e % c;
                        const uint64_t val = ((uint64_t)R[j * cs + lc].y << lb) | R[j * cs + lc].x;
                        if (!val) continue;
                        int g[kMaxVars];
                        bool ok = true;
                        for (int t = 0; t < nv; t++) {
                            g[t] = sU[t] + monoS[j * nv + t] - 1;
                            if (g[t] < 0) ok = false;
                        }
                        if (!ok) continue;  // cannot carry a coefficient on a valid path
                        const int h = dev_rank(g, nv, hdeg);
                        const int col = colmap[lc];
                        Hs[h * b + col] = addmod(Hs[h * b + col], val, I.Q.q);
                    }
                } else {
                    // move 2: store (first contribution) or add into the next phase's block
                    uint64_t *dst = nxt + (size_t)E.dest * s * b;
                    if (E.flags & 1u) {
                        for (int e = threadIdx.x; e < s * b; e += blockDim.x) dst[e] = 0;
                        __syncthreads();
                    }
                    for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
                        const int j = e / c, lc = e % c;
                        const uint64_t val = ((uint64_t)R[j * cs + lc].y << lb) | R[j * cs + lc].x;
                        uint64_t &slot = dst[(size_t)j * b + colmap[lc]];
                        slot = addmod(slot, val, I.Q.q);
                    }
                }
                __syncthreads();
            }
            __syncthreads();
        }
        uint64_t *out = Hout + (size_t)inst * h_stride;
        for (int e = threadIdx.x; e < (int)I.h_rows * b; e += blockDim.x) out[e] = Hs[e];
        __syncthreads();
    }
    if (false) {
    aborted:  // an MMA wait timed out: flag it, wait once more for the MMAs in flight, stop
        if (threadIdx.x == 0) atomicAdd(&counters[2], 1ull);
        if ((threadIdx.x & 127) == 0) mbar_wait(S.mbar[threadIdx.x >> 7], S.phase[threadIdx.x >> 7]);
        __syncthreads();
    }
    if (TC) tc_teardown(S.tmem);
    if (threadIdx.x == 0) {
        atomicAdd(&counters[0], my_chunks);
        atomicAdd(&counters[1], my_steps);
    }
}

}  // namespace zeta
#include "zeta_cluster.cuh"
#include "zeta_setup.cuh"
#include "zeta_large.cuh"
namespace zeta {

// Kernel-level Algorithm 2 on independent problems (zeta_horner_device):
// the same block routine as the chain kernel.
template <int CPT, bool MSMEM>
__global__ void __launch_bounds__(512) k_horner_problems(
    uint32_t count, int s, int c, const uint32_t *__restrict__ kk, const uint64_t *__restrict__ A,
    const uint64_t *__restrict__ B, uint64_t *__restrict__ W, const ModQ *__restrict__ mods,
    uint64_t *__restrict__ scratch) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t MASK30 = (1u << 30) - 1;
    unsigned char *ptr = smem_raw;
    uint64_t *Ms, *As;
    if (MSMEM) {
        Ms = (uint64_t *)ptr;
        As = Ms + (size_t)s * s;
        ptr += (size_t)2 * s * s * sizeof(uint64_t);
    } else {
        Ms = scratch + (size_t)blockIdx.x * 2 * s * s;
        As = Ms + (size_t)s * s;
    }
    uint2 *Wl = (uint2 *)ptr;
    uint2 *Vl = Wl + (size_t)s * pad4(c);
    const int cs = pad4(c);
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        const ModQ Q = mods[t];
        const int k = (int)kk[t];
        const uint64_t *At_g = A + (size_t)t * s * s;
        const uint64_t *Bt_g = B + (size_t)t * s * s;
        uint64_t *Wt = W + (size_t)t * s * c;
        for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
            const int r = e / s, j = e % s;  // row-major input
            const uint64_t a = to_mont(At_g[e], Q), b = to_mont(Bt_g[e], Q);
            As[(size_t)j * s + r] = a;
            Ms[(size_t)j * s + r] = addmod(mul_small(a, (uint64_t)(k > 0 ? k - 1 : 0), Q), b, Q.q);
        }
        for (int e = threadIdx.x; e < s * cs; e += blockDim.x) {
            const int j = e / cs, col = e - j * cs;
            const uint64_t w = col < c ? Wt[j * c + col] : 0;
            Wl[e] = make_uint2((uint32_t)w & MASK30, (uint32_t)(w >> 30));
        }
        __syncthreads();
        const int res = horner_block<CPT>(s, c, k, Ms, As, Wl, Vl, Q);
        const uint2 *R = res ? Vl : Wl;
        for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
            const int j = e / c, col = e - j * c;
            Wt[e] = ((uint64_t)R[j * cs + col].y << 30) | R[j * cs + col].x;
        }
        __syncthreads();
    }
}

// Kernel-level Algorithm 2 on independent problems with the limb-split GEMM
// steps on the tensor cores (s <= 64, c <= 16).  status[0] is set if an MMA
// wait timed out.
__global__ void __launch_bounds__(kTcThreads) k_horner_problems_tc(
    uint32_t count, int s, int c, const uint32_t *__restrict__ kk, const uint64_t *__restrict__ A,
    const uint64_t *__restrict__ B, uint64_t *__restrict__ W, const ModQ *__restrict__ mods,
    unsigned long long *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ uint2 s_ct[2 * kTcMaxL], s_ct_odd[2 * 16];
    __shared__ int s_abort[2];
    const uint32_t MASK30 = (1u << 30) - 1;
    const int sK = tc_sK(s), cs = pad4(c);
    TcState S;
    tc_carve(S, smem_raw, s);
    uint16_t *Aop = S.Aop;
    uint2 *Wl = reinterpret_cast<uint2 *>(smem_raw + tc_operand_bytes(s));
    uint2 *Vl = Wl + (size_t)s * cs;
    tc_setup(&s_tmem, s_mbar);
    S.ct_odd = s_ct_odd;
    S.tmem = s_tmem;
    S.mbar[0] = smem_u32(&s_mbar[0]);
    S.mbar[1] = smem_u32(&s_mbar[1]);
    S.phase[0] = S.phase[1] = 0;
    S.sK = sK;
    S.ct = s_ct;
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        const ModQ Q = mods[t];
        const int k = (int)kk[t];
        S.L = tc_digits(Q.q);
        tc_constants(Q, S.L, s_ct);
        const int kext = S.L * sK;
        uint32_t *a32 = reinterpret_cast<uint32_t *>(Aop);
        for (int e = threadIdx.x; e < 128 * kext / 2; e += blockDim.x) a32[e] = 0;
        __syncthreads();
        const uint64_t *At_g = A + (size_t)t * s * s;
        const uint64_t *Bt_g = B + (size_t)t * s * s;
        uint64_t *Wt = W + (size_t)t * s * c;
        for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
            const int r = e / s, j = e - r * s;  // row-major input
            const uint64_t a = At_g[e];
            const uint64_t x = addmod(mul_small(a, (uint64_t)(k > 0 ? k - 1 : 0), Q), Bt_g[e], Q.q);
            put_digits(Aop, 2 * r, j, sK, kext, S.L, x);
            put_digits(Aop, 2 * r + 1, j, sK, kext, S.L, a);
        }
        for (int e = threadIdx.x; e < s * cs; e += blockDim.x) {
            const int j = e / cs, col = e - j * cs;
            const uint64_t w = col < c ? Wt[j * c + col] : 0;
            Wl[e] = make_uint2((uint32_t)w & MASK30, (uint32_t)(w >> 30));
        }
        fence_async_smem();
        __syncthreads();
        const int res = horner_block_tc(S, s, c, k, Wl, Vl, Q, s_abort);
        if (res < 0) {
            if (threadIdx.x == 0) atomicOr(status, 1ull);
            // the MMAs in flight, bounded again
            if ((threadIdx.x & 127) == 0) mbar_wait(S.mbar[threadIdx.x >> 7], S.phase[threadIdx.x >> 7]);
            break;
        }
        const uint2 *R = res ? Vl : Wl;
        for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
            const int j = e / c, col = e - j * c;
            Wt[e] = ((uint64_t)R[j * cs + col].y << 30) | R[j * cs + col].x;
        }
        __syncthreads();
    }
    tc_teardown(S.tmem);
}

// Dynamic shared memory of k_horner_problems_tc.
inline size_t tc_problem_smem(int s, int c) {
    return tc_operand_bytes(s) + (size_t)2 * s * pad4(c) * sizeof(uint2);
}

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// A lane of the whole-GPU executor: its own stream and buffers, so that several instances run at once, one host
// thread each.  Slot 0 uses the engine's stream.
struct LgSlot {
    cudaStream_t stream = nullptr;
    bool owned = false;
    std::map<std::string, DevBuf> bufs;
};

struct DeviceEngine {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;  // second lane for pipelined sub-batches (non-blocking, created on first use)
    int sms = 0;
    std::map<std::string, DevBuf> bufs;
    std::vector<LgSlot> lg;       // whole-GPU executor lanes (created on first use)
    bool binom_ready = false;
};

static zeta_status ensure_in(std::map<std::string, DevBuf> &bufs, const char *name, size_t bytes, void **out,
                             std::string &err) {
    DevBuf &b = bufs[name];
    if (b.bytes < bytes) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        size_t want = std::max(bytes, (size_t)256);
        cudaError_t ce = cudaMalloc(&b.ptr, want);
        if (ce != cudaSuccess) {
            err = std::string("cudaMalloc ") + name + ": " + cudaGetErrorString(ce);
            cudaGetLastError();
            return ZETA_ERR_OOM;
        }
        b.bytes = want;
    }
    *out = b.ptr;
    return ZETA_OK;
}

static zeta_status ensure(DeviceEngine *e, const char *name, size_t bytes, void **out, std::string &err) {
    return ensure_in(e->bufs, name, bytes, out, err);
}

static ModQ make_modq(uint64_t q) {
    ModQ Q;
    Q.q = q;
    uint64_t inv = 1;
    for (int i = 0; i < 7; i++) inv *= 2 - q * inv;
    Q.qneg_inv = (uint64_t)0 - inv;
    u128 R = ((u128)1 << 64) % q;
    Q.r2 = (uint64_t)(R * R % q);
    Q.k30 = (uint64_t)((R << 30) % q);
    return Q;
}

DeviceEngine *engine_create(int device, void *stream, std::string &err) {
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0) {
        err = std::string("no CUDA device: ") + cudaGetErrorString(ce);
        cudaGetLastError();
        return nullptr;
    }
    if (device < 0 || device >= ndev) { err = "device index out of range"; return nullptr; }
    ce = cudaSetDevice(device);
    if (ce != cudaSuccess) { err = cudaGetErrorString(ce); return nullptr; }
    DeviceEngine *e = new (std::nothrow) DeviceEngine();
    if (!e) { err = "host allocation"; return nullptr; }
    e->device = device;
    e->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, device);
    return e;
}

int engine_sm_count(const DeviceEngine *e) { return e ? e->sms : 0; }

void engine_destroy(DeviceEngine *e) {
    if (!e) return;
    cudaSetDevice(e->device);
    if (e->side) cudaStreamDestroy(e->side);
    for (auto &kv : e->bufs)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    for (LgSlot &sl : e->lg) {
        if (sl.owned && sl.stream) cudaStreamDestroy(sl.stream);
        for (auto &kv : sl.bufs)
            if (kv.second.ptr) cudaFree(kv.second.ptr);
    }
    delete e;
}

static zeta_status upload_binom(DeviceEngine *e, std::string &err) {
    if (e->binom_ready) return ZETA_OK;
    static int32_t h[64][9];
    for (int a = 0; a < 64; a++)
        for (int b = 0; b < 9; b++) {
            long long r = 1;
            if (b > a) r = 0;
            else for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
            h[a][b] = (int32_t)r;
        }
    CUDA_TRY(cudaMemcpyToSymbol(c_binom, h, sizeof(h)));
    e->binom_ready = true;
    return ZETA_OK;
}

template <typename T>
static zeta_status upload(DeviceEngine *e, const char *name, const std::vector<T> &v, T **out, std::string &err) {
    void *p;
    zeta_status st = ensure(e, name, sizeof(T) * std::max<size_t>(v.size(), 1), &p, err);
    if (st) return st;
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, e->stream));
    *out = (T *)p;
    return ZETA_OK;
}

template <typename T>
static zeta_status upload_in(LgSlot &sl, const char *name, const std::vector<T> &v, T **out, std::string &err) {
    void *p;
    zeta_status st = ensure_in(sl.bufs, name, sizeof(T) * std::max<size_t>(v.size(), 1), &p, err);
    if (st) return st;
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, sl.stream));
    *out = (T *)p;
    return ZETA_OK;
}

struct DeviceBatch {
    cudaStream_t stream = nullptr;  // the lane every upload, launch and download of this batch uses
    std::vector<Instance *> insts;
    zeta_policy policy;
    zeta_path path;
    std::vector<void *> allocs;
    DInst *d_inst = nullptr;
    DTab *d_tabs = nullptr;
    int32_t *d_tabpool = nullptr;
    uint64_t *d_sec = nullptr;
    DChain *d_chains = nullptr;
    Term *d_terms = nullptr;
    uint32_t *d_phases = nullptr;
    DEntry *d_entries = nullptr;
    DChunk *d_chunks = nullptr;
    uint32_t *d_order = nullptr, *d_queue = nullptr;
    uint64_t *d_scratch = nullptr, *d_blocks = nullptr, *d_H = nullptr;
    unsigned long long *d_counters = nullptr;
    unsigned long long *d_stamps = nullptr;  // 2 per instance + the launch start (device latency)
    int grid = 1, threads = 256;
    bool msmem = true;
    bool tc = false;
    bool cluster = false;      // k_execute_cluster (instances with s > kClusterMinS)
    int cl = 1;                // CTAs per cluster
    int smax = 0, cmax = 0;    // largest s and b of the batch (cluster shared-memory carve)
    size_t smem = 0, scratch_stride = 0, blocks_stride = 0, h_stride = 0;
    uint64_t bytes = 0, bytes_h2d = 0, bytes_d2h = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;  // around each recurrence launch
    cudaGraphExec_t graph_exec = nullptr;                      // captured launches of one run
    cudaStream_t cap_stream = nullptr;
    double ms_kernel = 0;
    uint64_t launches = 0;
};

template <typename T>
static zeta_status dev_alloc(DeviceBatch *B, size_t count, T **out, std::string &err) {
    void *p = nullptr;
    size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
    cudaError_t ce = cudaMalloc(&p, bytes);
    if (ce != cudaSuccess) {
        err = std::string("cudaMalloc: ") + cudaGetErrorString(ce);
        cudaGetLastError();
        return ZETA_ERR_OOM;
    }
    B->allocs.push_back(p);
    B->bytes += bytes;
    *out = (T *)p;
    return ZETA_OK;
}

template <typename T>
static zeta_status dev_upload(DeviceEngine *e, DeviceBatch *B, const std::vector<T> &v, T **out, std::string &err) {
    zeta_status st = dev_alloc(B, v.size(), out, err);
    if (st) return st;
    (void)e;
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, B->stream));
    B->bytes_h2d += sizeof(T) * v.size();
    return ZETA_OK;
}

void engine_release(DeviceBatch *B) {
    if (!B) return;
    if (B->graph_exec) cudaGraphExecDestroy(B->graph_exec);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    for (auto &ev : B->events) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    for (void *p : B->allocs) cudaFree(p);
    delete B;
}

void engine_batch_timing(const DeviceBatch *B, double *ms_kernel, uint64_t *launches, uint64_t *h2d, uint64_t *d2h) {
    if (!B) { *ms_kernel = 0; *launches = 0; *h2d = 0; *d2h = 0; return; }
    *ms_kernel = B->ms_kernel;
    *launches = B->launches;
    *h2d = B->bytes_h2d;
    *d2h = B->bytes_d2h;
}

zeta_status engine_prepare(DeviceEngine *e, std::vector<Instance *> &batch, zeta_policy policy, zeta_path path,
                           uint32_t block_threads, int lane, DeviceBatch **out, std::string &err) {
    *out = nullptr;
    CUDA_TRY(cudaSetDevice(e->device));
    zeta_status st = upload_binom(e, err);
    if (st) return st;
    if (lane && !e->side) CUDA_TRY(cudaStreamCreateWithFlags(&e->side, cudaStreamNonBlocking));
    DeviceBatch *B = new (std::nothrow) DeviceBatch();
    if (!B) return ZETA_ERR_OOM;
    B->stream = lane ? e->side : e->stream;
    B->insts = batch;
    B->policy = policy;
    B->path = path;

    std::map<uint64_t, uint32_t> tab_of;  // (n, d, S) -> table set
    std::vector<DTab> tabs;
    std::vector<int32_t> tabpool;
    std::vector<DInst> dinst;
    std::vector<uint64_t> secpool;
    std::vector<DChain> dchains;
    std::vector<Term> dterms;
    std::vector<uint32_t> phases;
    std::vector<DEntry> dentries;
    std::vector<DChunk> dchunks;
    std::vector<uint64_t> work(batch.size());
    int max_s = 0, max_c = 0, max_h = 0;
    size_t max_block_words = 0;
    for (size_t ii = 0; ii < batch.size(); ii++) {
        Instance *X = batch[ii];
        const uint64_t key = ((uint64_t)X->n << 48) | ((uint64_t)X->d << 32) | X->Smask;
        if (!tab_of.count(key)) {
            // index tables built by the host setup (they depend on n, d and S only):
            // monoS = mu + 1 - 1_S, secrow[i][omega] = row (i, omega - 1_S + e_i) of Sec or -1.
            // The kernel reads them with the formulas of S = {0..n}; with the section of J_S
            // and the shifted exponents those are Prop. 3.3 for the instance's S.
            DTab T;
            T.nv = X->nv;
            T.s = X->s;
            T.h_rows = X->h_rows;
            T.monoS_off = (uint32_t)tabpool.size();
            tabpool.insert(tabpool.end(), X->tab_monoS.begin(), X->tab_monoS.end());
            T.secrow_off = (uint32_t)tabpool.size();
            tabpool.insert(tabpool.end(), X->tab_secrow.begin(), X->tab_secrow.end());
            tab_of[key] = (uint32_t)tabs.size();
            tabs.push_back(T);
        }
        DInst I;
        std::memset(&I, 0, sizeof(I));
        I.Q = make_modq(X->q);
        I.n = X->n; I.d = X->d; I.b = X->b; I.s = X->s; I.nv = X->nv;
        I.sec_rows = X->sec_rows; I.sec_cols = X->sec_cols; I.h_rows = X->h_rows; I.kappa = X->kappa;
        I.tab = tab_of[key];
        I.sec_off = secpool.size();
        {
            // Sec R mod q: the step matrices built from it are in Montgomery form
            const u128 Rm = ((u128)1 << 64) % X->q;
            for (uint64_t v : X->sec) secpool.push_back((uint64_t)((u128)v * Rm % X->q));
        }
        I.chain_base = (uint32_t)dchains.size();
        I.chunk_base = (uint32_t)dchunks.size();
        I.phase_off = (uint32_t)phases.size();
        I.nphases = (uint32_t)X->plan.phase_begin.size() - 1;
        uint32_t ebase = (uint32_t)dentries.size();
        for (uint32_t pb : X->plan.phase_begin) phases.push_back(ebase + pb);
        for (const PlanEntry &pe : X->plan.entries) {
            DEntry de;
            std::memcpy(de.U, pe.U, sizeof(de.U));
            de.chunk_begin = pe.chunk_begin;
            de.chunk_end = pe.chunk_end;
            de.arrival = pe.arrival;
            de.start_chain = pe.start_chain;
            de.dest = pe.dest;
            de.flags = pe.flags;
            de.live = (uint32_t)pe.live;  // b <= 32 on the persistent executors
            dentries.push_back(de);
        }
        for (const PlanChunk &pc : X->plan.chunks) {
            DChunk dc;
            std::memcpy(dc.v, pc.v, sizeof(dc.v));
            dc.k = pc.k;
            dchunks.push_back(dc);
        }
        dinst.push_back(I);
        max_s = std::max(max_s, (int)X->s);
        max_c = std::max(max_c, (int)X->b);
        max_h = std::max(max_h, (int)X->h_rows);
        max_block_words = std::max(max_block_words, (size_t)X->plan.cap * X->s * X->b);
        uint32_t tbase = (uint32_t)dterms.size();
        for (auto &ch : X->chains) {
            DChain dc;
            std::memcpy(dc.U, ch.U, sizeof(dc.U));
            dc.term_begin = ch.term_begin + tbase;
            dc.term_end = ch.term_end + tbase;
            dchains.push_back(dc);
        }
        dterms.insert(dterms.end(), X->terms.begin(), X->terms.end());
        work[ii] = X->plan.work + (uint64_t)X->plan.chunks.size() * X->s * X->s * 8;
    }
    if (max_s > kMaxS || max_c > kMaxC) {
        err = "instance too large for the device kernels";
        engine_release(B);
        return ZETA_ERR_UNSUPPORTED;
    }
    // instances in decreasing work (longest-processing-time order for the persistent queue)
    std::vector<uint32_t> order(batch.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (uint32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return work[a] > work[b]; });
#define UP(vec, ptr) if ((st = dev_upload(e, B, vec, &B->ptr, err))) { engine_release(B); return st; }
    UP(dinst, d_inst);
    UP(tabs, d_tabs);
    UP(tabpool, d_tabpool);
    const bool use_cluster = path == ZETA_PATH_VECTOR && max_s > kClusterMinS;
    if (use_cluster) {
        // the cluster executor reads each section column gamma as one contiguous run of rows (i, nu)
        std::vector<uint64_t> secT(secpool.size());
        for (size_t ii = 0; ii < batch.size(); ii++) {
            const DInst &I = dinst[ii];
            for (uint32_t r = 0; r < I.sec_rows; r++)
                for (uint32_t c = 0; c < I.sec_cols; c++)
                    secT[I.sec_off + (size_t)c * I.sec_rows + r] = secpool[I.sec_off + (size_t)r * I.sec_cols + c];
        }
        secpool.swap(secT);
    }
    UP(secpool, d_sec);
    UP(dchains, d_chains);
    UP(dterms, d_terms);
    UP(phases, d_phases);
    UP(dentries, d_entries);
    UP(dchunks, d_chunks);
    UP(order, d_order);
#undef UP
    if (path != ZETA_PATH_VECTOR && path != ZETA_PATH_GEMM) {
        err = "unknown path";
        engine_release(B);
        return ZETA_ERR_ARG;
    }
    if (path == ZETA_PATH_GEMM && (max_s > kTcMaxS || max_c > kTcMaxC)) {
        err = "the tensor-core path takes s <= 64 and b <= 16";
        engine_release(B);
        return ZETA_ERR_UNSUPPORTED;
    }
    B->tc = path == ZETA_PATH_GEMM;
    B->smax = max_s;
    B->cmax = max_c;
    const void *kfn;
    if (use_cluster) {
        // the smallest cluster whose CTAs hold their rows of M and both W buffers in shared memory, for every
        // instance of the batch
        auto need = [&](int cl, size_t *a_words) {
            size_t bytes = 0, aw = 0;
            for (Instance *X : batch) {
                const int R = ((int)X->s + cl - 1) / cl;
                bytes = std::max(bytes, cl_smem((int)X->s, (int)X->b, R));
                aw = std::max(aw, (size_t)R * X->s);
            }
            if (a_words) *a_words = aw;
            return bytes;
        };
        int cl = 1;
        while (cl <= 16 && need(cl, nullptr) > (size_t)220 * 1024) cl *= 2;
        if (cl > 16) {
            err = "step matrices too large for a cluster of 16 CTAs";
            engine_release(B);
            return ZETA_ERR_UNSUPPORTED;
        }
        size_t a_words = 0;
        B->cluster = true;
        B->cl = cl;
        B->smem = need(cl, &a_words);
        B->msmem = true;
        B->threads = kClThreads;
        kfn = (const void *)k_execute_cluster;
        CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem));
        if (cl > 8) CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(cl * e->sms));
        cfg.blockDim = dim3((unsigned)B->threads);
        cfg.dynamicSmemBytes = B->smem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, kfn, &cfg));
        if (nclusters < 1) {
            err = "no cluster of this size fits an SM group";
            engine_release(B);
            return ZETA_ERR_UNSUPPORTED;
        }
        nclusters = (int)std::min<size_t>((size_t)nclusters, batch.size());
        B->grid = nclusters * cl;
        B->scratch_stride = (a_words + 1) & ~(size_t)1;  // this CTA's rows of A (16-byte aligned)
        B->blocks_stride = 2 * std::max<size_t>(max_block_words, 1);
        B->h_stride = (size_t)max_h * max_c;
#define AL(count, ptr) if ((st = dev_alloc(B, count, &B->ptr, err))) { engine_release(B); return st; }
        AL(B->scratch_stride * B->grid, d_scratch);
        AL(B->blocks_stride * nclusters, d_blocks);
        AL(B->h_stride * batch.size(), d_H);
        AL(16, d_queue);
        AL(8, d_counters);
        AL(2 * batch.size() + 1, d_stamps);
#undef AL
        *out = B;
        return ZETA_OK;
    }
    if (B->tc) {
        // Ms/As are replaced by the GEMM operands; at most two blocks per SM
        // (their accumulators fill the 512 TMEM columns)
        B->smem = tc_operand_bytes(max_s) + chain_smem(max_s, max_c, max_h) - (size_t)2 * max_s * max_s * 8 *
                                                                                  (mats_in_smem(max_s) ? 1 : 0);
        B->msmem = false;
        B->threads = kTcThreads;
        kfn = (const void *)k_execute<4, false, true>;
    } else {
        B->smem = chain_smem(max_s, max_c, max_h);
        B->msmem = mats_in_smem(max_s);
        B->threads = launch_threads(max_s, max_c);
        if (block_threads) {
            if (block_threads % 32 || block_threads < 64 || block_threads > 512) {
                err = "block_threads must be a multiple of 32 in [64, 512]";
                engine_release(B);
                return ZETA_ERR_ARG;
            }
            B->threads = (int)block_threads;
        }
        kfn = B->msmem ? (const void *)k_execute<4, true, false> : (const void *)k_execute<4, false, false>;
    }
    CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, B->threads, B->smem));
    per_sm = std::max(1, per_sm);
    if (B->tc) per_sm = std::min(per_sm, 2);
    B->grid = std::max(1, (int)std::min<size_t>((size_t)e->sms * per_sm, batch.size()));
    // the tensor-core kernel reads the largest s of the batch from this argument
    B->scratch_stride = B->tc ? (size_t)max_s : (size_t)2 * max_s * max_s;
    B->blocks_stride = 2 * std::max<size_t>(max_block_words, 1);
    B->h_stride = (size_t)max_h * max_c;
#define AL(count, ptr) if ((st = dev_alloc(B, count, &B->ptr, err))) { engine_release(B); return st; }
    AL((B->msmem || B->tc) ? 1 : B->scratch_stride * B->grid, d_scratch);
    AL(B->blocks_stride * B->grid, d_blocks);
    AL(B->h_stride * batch.size(), d_H);
    AL(16, d_queue);
    AL(8, d_counters);
    AL(2 * batch.size() + 1, d_stamps);
#undef AL
    *out = B;
    return ZETA_OK;
}

// Enqueue one run of the batch (counter resets and the persistent kernel) on `st`.
static cudaError_t enqueue_batch(DeviceBatch *B, cudaStream_t st) {
    cudaError_t ce = cudaMemsetAsync(B->d_queue, 0, 16 * sizeof(uint32_t), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(B->d_counters, 0, 8 * sizeof(unsigned long long), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(B->d_stamps, 0, 2 * B->insts.size() * sizeof(unsigned long long), st);
    if (ce == cudaSuccess)
        ce = cudaMemsetAsync(B->d_stamps + 2 * B->insts.size(), 0xff, sizeof(unsigned long long), st);
    if (ce != cudaSuccess) return ce;
#define LAUNCH(MS, TC)                                                                                      \
    k_execute<4, MS, TC><<<B->grid, B->threads, B->smem, st>>>(                                             \
        B->d_inst, B->d_tabs, B->d_tabpool, B->d_sec, B->d_chains, B->d_terms, B->d_phases, B->d_entries,    \
        B->d_chunks, B->d_order, (uint32_t)B->insts.size(), B->d_queue, B->d_scratch, B->scratch_stride,     \
        B->d_blocks, B->blocks_stride, B->d_H, B->h_stride, B->d_counters, B->d_stamps)
    if (B->cluster) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = B->cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)B->grid);
        cfg.blockDim = dim3((unsigned)B->threads);
        cfg.dynamicSmemBytes = B->smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ce = cudaLaunchKernelEx(&cfg, k_execute_cluster, (const DInst *)B->d_inst, (const DTab *)B->d_tabs,
                                (const int32_t *)B->d_tabpool, (const uint64_t *)B->d_sec, (const DChain *)B->d_chains,
                                (const Term *)B->d_terms, (const uint32_t *)B->d_phases,
                                (const DEntry *)B->d_entries, (const DChunk *)B->d_chunks,
                                (const uint32_t *)B->d_order, (uint32_t)B->insts.size(), B->d_queue, B->d_scratch,
                                B->scratch_stride, B->d_blocks, B->blocks_stride, B->d_H, B->h_stride,
                                B->d_counters, B->d_stamps);
        if (ce != cudaSuccess) return ce;
    }
    else if (B->tc) LAUNCH(false, true);
    else if (B->msmem) LAUNCH(true, false);
    else LAUNCH(false, false);
#undef LAUNCH
    return cudaGetLastError();
}

// The first run of a prepared batch captures its launches into a CUDA graph
// (on a private stream, so that the caller's stream may be the legacy default
// stream); every run replays the graph on the engine's stream.
zeta_status engine_launch(DeviceEngine *e, DeviceBatch *B, std::string &err) {
    CUDA_TRY(cudaSetDevice(e->device));
    if (!B->graph_exec) {
        if (!B->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
        CUDA_TRY(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t ce = enqueue_batch(B, B->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t ce2 = cudaStreamEndCapture(B->cap_stream, &g);
        if (ce != cudaSuccess || ce2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            err = std::string("graph capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ce2);
            cudaGetLastError();
            return ZETA_ERR_DEVICE;
        }
        const cudaError_t ce3 = cudaGraphInstantiate(&B->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ce3 != cudaSuccess) {
            B->graph_exec = nullptr;
            err = std::string("graph instantiate: ") + cudaGetErrorString(ce3);
            cudaGetLastError();
            return ZETA_ERR_DEVICE;
        }
    }
    cudaEvent_t ev0, ev1;
    CUDA_TRY(cudaEventCreate(&ev0));
    CUDA_TRY(cudaEventCreate(&ev1));
    B->events.push_back({ev0, ev1});
    CUDA_TRY(cudaEventRecord(ev0, B->stream));
    CUDA_TRY(cudaGraphLaunch(B->graph_exec, B->stream));
    CUDA_TRY(cudaEventRecord(ev1, B->stream));
    return ZETA_OK;
}

zeta_status engine_collect(DeviceEngine *e, DeviceBatch *B, std::string &err) {
    CUDA_TRY(cudaSetDevice(e->device));
    std::vector<uint64_t> hH(B->h_stride * B->insts.size());
    unsigned long long hc[8] = {0};
    CUDA_TRY(cudaMemcpyAsync(hH.data(), B->d_H, sizeof(uint64_t) * hH.size(), cudaMemcpyDeviceToHost, B->stream));
    CUDA_TRY(cudaMemcpyAsync(hc, B->d_counters, sizeof(hc), cudaMemcpyDeviceToHost, B->stream));
    std::vector<unsigned long long> hs(2 * B->insts.size() + 1);
    CUDA_TRY(cudaMemcpyAsync(hs.data(), B->d_stamps, sizeof(unsigned long long) * hs.size(), cudaMemcpyDeviceToHost,
                             B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    B->bytes_d2h = sizeof(uint64_t) * hH.size();
    B->ms_kernel = 0;
    B->launches = 0;
    for (auto &ev : B->events) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev.first, ev.second);
        B->ms_kernel += ms;
        B->launches++;
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    B->events.clear();
    uint64_t played = 0;
    for (size_t ii = 0; ii < B->insts.size(); ii++) {
        Instance *X = B->insts[ii];
        X->H.assign(hH.begin() + ii * B->h_stride, hH.begin() + ii * B->h_stride + (size_t)X->h_rows * X->b);
        X->steps = X->plan.steps;
        X->column_steps = X->plan.column_steps;
        X->chunks = X->plan.chunks_played;
        played += X->plan.chunks_played;
        const unsigned long long t0 = hs[2 * B->insts.size()];
        X->ms_dev_start = hs[2 * ii] >= t0 ? (hs[2 * ii] - t0) * 1e-6 : 0.0;
        X->ms_dev_end = hs[2 * ii + 1] >= t0 ? (hs[2 * ii + 1] - t0) * 1e-6 : 0.0;
    }
    if (hc[2]) {
        err = "a tensor-core step timed out";
        return ZETA_ERR_TIMEOUT;
    }
    if (hc[0] != played) {  // counters are reset by every launch
        err = "device played a different number of chunks than planned";
        return ZETA_ERR_INTERNAL;
    }
    return ZETA_OK;
}

zeta_status engine_run(DeviceEngine *e, std::vector<Instance *> &batch, zeta_policy policy, zeta_path path,
                       uint32_t block_threads, std::string &err, double *ms_device) {
    cudaEvent_t ev0, ev1;
    CUDA_TRY(cudaSetDevice(e->device));
    CUDA_TRY(cudaEventCreate(&ev0));
    CUDA_TRY(cudaEventCreate(&ev1));
    CUDA_TRY(cudaEventRecord(ev0, e->stream));
    DeviceBatch *B = nullptr;
    zeta_status st = engine_prepare(e, batch, policy, path, block_threads, 0, &B, err);
    if (!st) st = engine_launch(e, B, err);
    if (!st) st = engine_collect(e, B, err);
    cudaEventRecord(ev1, e->stream);
    cudaEventSynchronize(ev1);
    float ms = 0;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (ms_device) *ms_device = ms;
    engine_release(B);
    return st;
}

zeta_status engine_horner(DeviceEngine *e, zeta_path path, uint32_t count, uint32_t s, uint32_t c,
                          const uint32_t *k, const uint64_t *A, const uint64_t *B, uint64_t *W,
                          const uint64_t *q, std::string &err) {
    CUDA_TRY(cudaSetDevice(e->device));
    if (s == 0 || c == 0 || s > kMaxS || c > kMaxC) { err = "s or c out of range"; return ZETA_ERR_ARG; }
    if (path == ZETA_PATH_GEMM && (s > (uint32_t)kTcMaxS || c > (uint32_t)kTcMaxC)) {
        err = "the tensor-core path takes s <= 64 and c <= 16";
        return ZETA_ERR_ARG;
    }
    if (path != ZETA_PATH_VECTOR && path != ZETA_PATH_GEMM) { err = "unknown path"; return ZETA_ERR_ARG; }
    if (count == 0) return ZETA_OK;
    std::vector<uint64_t> hq(count);
    CUDA_TRY(cudaMemcpy(hq.data(), q, sizeof(uint64_t) * count, cudaMemcpyDeviceToHost));
    std::vector<ModQ> mods(count);
    for (uint32_t t = 0; t < count; t++) {
        if (hq[t] < 2 || hq[t] > ((uint64_t)1 << 60) || !(hq[t] & 1) || (uint64_t)s >= 8 * hq[t]) {
            err = "modulus must be odd, in [3, 2^60] and above s/8";
            return ZETA_ERR_ARG;
        }
        mods[t] = make_modq(hq[t]);
    }
    ModQ *d_mods;
    zeta_status st = upload(e, "hmods", mods, &d_mods, err);
    if (st) return st;
    if (path == ZETA_PATH_GEMM) {
        unsigned long long *d_status;
        if ((st = ensure(e, "hstatus", sizeof(unsigned long long), (void **)&d_status, err))) return st;
        const size_t smem = tc_problem_smem((int)s, (int)c);
        CUDA_TRY(cudaFuncSetAttribute((const void *)k_horner_problems_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        int per_sm = 0;
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_horner_problems_tc, kTcThreads,
                                                               smem));
        per_sm = std::max(1, std::min(per_sm, 2));  // two blocks' accumulators fill the 512 TMEM columns
        const int grid = (int)std::min<uint32_t>(count, (uint32_t)(e->sms * per_sm));
        CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(unsigned long long), e->stream));
        k_horner_problems_tc<<<grid, kTcThreads, smem, e->stream>>>(count, (int)s, (int)c, k, A, B, W, d_mods,
                                                                     d_status);
        CUDA_TRY(cudaGetLastError());
        unsigned long long flag = 0;
        CUDA_TRY(cudaMemcpyAsync(&flag, d_status, sizeof(flag), cudaMemcpyDeviceToHost, e->stream));
        CUDA_TRY(cudaStreamSynchronize(e->stream));
        if (flag) { err = "tensor-core step timed out"; return ZETA_ERR_TIMEOUT; }
        return ZETA_OK;
    }
    int grid = (int)std::min<uint32_t>(count, (uint32_t)e->sms * 4);
    uint64_t *d_scratch;
    if ((st = ensure(e, "hscratch", sizeof(uint64_t) * 2 * s * s * (size_t)grid, (void **)&d_scratch, err))) return st;
    const bool ms = mats_in_smem((int)s);
    size_t smem = (size_t)2 * s * pad4((int)c) * sizeof(uint2) + (ms ? (size_t)2 * s * s * sizeof(uint64_t) : 0);
    const int threads = launch_threads((int)s, (int)c);
    const void *kfn = ms ? (const void *)k_horner_problems<4, true> : (const void *)k_horner_problems<4, false>;
    CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ms) k_horner_problems<4, true><<<grid, threads, smem, e->stream>>>(count, (int)s, (int)c, k, A, B, W, d_mods, d_scratch);
    else k_horner_problems<4, false><<<grid, threads, smem, e->stream>>>(count, (int)s, (int)c, k, A, B, W, d_mods, d_scratch);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(e->stream));
    return ZETA_OK;
}


// Right inverses of the host setup on the device (k_right_inverse, one block per job).  A job whose
// pivot row (C + R words) does not fit the block's shared memory is left for the host.
zeta_status engine_solve(DeviceEngine *e, const std::vector<SolveJob *> &jobs, const std::vector<uint64_t> &qs,
                         const std::vector<uint64_t> &ps, std::string &err, double *ms_device) {
    if (ms_device) *ms_device = 0;
    if (jobs.size() != qs.size() || jobs.size() != ps.size()) { err = "engine_solve: sizes differ"; return ZETA_ERR_ARG; }
    CUDA_TRY(cudaSetDevice(e->device));
    int max_smem = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->device));
    std::vector<SolveDesc> descs;
    std::vector<SolveJob *> mine;
    std::vector<uint32_t> nz_idx;
    std::vector<uint64_t> nz_val;
    uint64_t work = 0, outw = 0;
    uint32_t npiv = 0, maxW = 0;
    for (size_t t = 0; t < jobs.size(); t++) {
        SolveJob &J = *jobs[t];
        if (J.done || J.R <= 0 || J.C <= 0) continue;
        const uint64_t W = (uint64_t)J.C + (uint64_t)J.R;
        if (W * sizeof(uint64_t) > (uint64_t)max_smem || (uint64_t)J.R * (uint64_t)J.C >= ((uint64_t)1 << 32)) continue;
        if (J.A.size() != (size_t)J.R * J.C || qs[t] < 3 || !(qs[t] & 1) || qs[t] >= ((uint64_t)1 << 60) || ps[t] < 2) {
            err = "engine_solve: malformed job";
            return ZETA_ERR_ARG;
        }
        SolveDesc d;
        std::memset(&d, 0, sizeof(d));
        d.Q = make_modq(qs[t]);
        d.p = ps[t];
        d.aug = work;
        d.out = outw;
        d.nz = nz_idx.size();
        for (size_t x = 0; x < J.A.size(); x++)
            if (J.A[x]) {
                nz_idx.push_back((uint32_t)x);
                nz_val.push_back(J.A[x]);
            }
        d.nnz = (uint32_t)(nz_idx.size() - d.nz);
        d.R = (uint32_t)J.R;
        d.C = (uint32_t)J.C;
        d.W = (uint32_t)W;
        d.piv = npiv;
        work += (uint64_t)J.R * W;
        outw += (uint64_t)J.R * J.R;
        npiv += (uint32_t)J.R;
        maxW = std::max(maxW, (uint32_t)W);
        descs.push_back(d);
        mine.push_back(&J);
    }
    if (descs.empty()) return ZETA_OK;
    const uint32_t count = (uint32_t)descs.size();
    // a few matrices with R >= 1000 rows (a cubic threefold's section, a cubic fourfold's section and its final
    // level m = 5) take the whole GPU, one at a time; the others, or many large ones, one block each in a single
    // launch
    uint32_t nlarge = 0;
    for (const SolveDesc &d : descs) nlarge += d.R >= 1000;
    std::vector<SolveDesc> small_descs;
    std::vector<uint32_t> small_of, big_of;
    for (uint32_t t = 0; t < count; t++) {
        if (descs[t].R >= 1000 && nlarge <= 8) big_of.push_back(t);
        else {
            small_of.push_back(t);
            small_descs.push_back(descs[t]);
        }
    }
    SolveDesc *d_desc;
    uint32_t *d_idx;
    uint64_t *d_val, *d_work, *d_out;
    int32_t *d_piv, *d_rank;
    SolveState *d_state;
    zeta_status st;
    if ((st = upload(e, "sv_desc", small_descs, &d_desc, err))) return st;
    if ((st = upload(e, "sv_idx", nz_idx, &d_idx, err))) return st;
    if ((st = upload(e, "sv_val", nz_val, &d_val, err))) return st;
    if ((st = ensure(e, "sv_work", sizeof(uint64_t) * work, (void **)&d_work, err))) return st;
    if ((st = ensure(e, "sv_out", sizeof(uint64_t) * outw, (void **)&d_out, err))) return st;
    if ((st = ensure(e, "sv_piv", sizeof(int32_t) * npiv, (void **)&d_piv, err))) return st;
    if ((st = ensure(e, "sv_rank", sizeof(int32_t) * count, (void **)&d_rank, err))) return st;
    if ((st = ensure(e, "sv_state", sizeof(SolveState), (void **)&d_state, err))) return st;
    const size_t smem = (size_t)maxW * sizeof(uint64_t);
    CUDA_TRY(cudaFuncSetAttribute((const void *)k_right_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUDA_TRY(cudaFuncSetAttribute((const void *)k_ri_elim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_right_inverse, kSolveThreads, smem));
    cudaEvent_t ev[2];
    CUDA_TRY(cudaEventCreate(&ev[0]));
    CUDA_TRY(cudaEventCreate(&ev[1]));
    cudaEventRecord(ev[0], e->stream);
    cudaError_t le = cudaSuccess;
    if (!small_of.empty()) {
        const int grid = (int)std::min<uint64_t>(small_of.size(), (uint64_t)e->sms * std::max(per_sm, 1));
        k_right_inverse<<<grid, kSolveThreads, smem, e->stream>>>(d_desc, (uint32_t)small_of.size(), d_idx, d_val,
                                                                  d_work, d_out, d_piv, d_rank);
        le = cudaGetLastError();
    }
    for (size_t b = 0; b < big_of.size() && le == cudaSuccess; b++) {
        const SolveDesc &D = descs[big_of[b]];
        const size_t words = (size_t)D.R * D.W;
        const unsigned fill_grid = (unsigned)std::min<size_t>((words + 1023) / 1024, (size_t)e->sms * 8);
        const size_t esmem = (size_t)D.W * sizeof(uint64_t);
        int elim_per_sm = 0;
        le = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&elim_per_sm, (const void *)k_ri_elim, kSolveThreads, esmem);
        if (le != cudaSuccess) break;
        const unsigned elim_grid = (unsigned)std::min<int64_t>((D.R + 15) / 16, (int64_t)e->sms * std::max(elim_per_sm, 1));
        k_ri_init<<<fill_grid, 1024, 0, e->stream>>>(D, d_idx, d_val, d_work, d_state);
        if (D.nnz) k_ri_scatter<<<(D.nnz + 1023) / 1024, 1024, 0, e->stream>>>(D, d_idx, d_val, d_work);
        for (uint32_t c = 0; c < D.C; c++) {
            k_ri_pivot<<<1, 1024, 0, e->stream>>>(D, (int)c, d_work, d_piv, d_state);
            k_ri_elim<<<elim_grid, kSolveThreads, esmem, e->stream>>>(D, (int)c, d_work, d_state);
        }
        k_ri_out<<<(unsigned)e->sms * 4, 256, 0, e->stream>>>(D, d_work, d_out, d_state, d_rank + small_of.size() + b);
        le = cudaGetLastError();
    }
    if (le == cudaSuccess) le = cudaEventRecord(ev[1], e->stream);
    std::vector<uint64_t> out(outw);
    std::vector<int32_t> piv(npiv), rank_dev(count);
    if (le == cudaSuccess) {
        le = cudaMemcpyAsync(out.data(), d_out, sizeof(uint64_t) * outw, cudaMemcpyDeviceToHost, e->stream);
        if (le == cudaSuccess) le = cudaMemcpyAsync(piv.data(), d_piv, sizeof(int32_t) * npiv, cudaMemcpyDeviceToHost, e->stream);
        if (le == cudaSuccess) le = cudaMemcpyAsync(rank_dev.data(), d_rank, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, e->stream);
        if (le == cudaSuccess) le = cudaStreamSynchronize(e->stream);
    }
    float ms = 0;
    if (le == cudaSuccess) cudaEventElapsedTime(&ms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    CUDA_TRY(le);
    if (ms_device) *ms_device = ms;
    std::vector<int32_t> rank(count);
    for (size_t i = 0; i < small_of.size(); i++) rank[small_of[i]] = rank_dev[i];
    for (size_t b = 0; b < big_of.size(); b++) rank[big_of[b]] = rank_dev[small_of.size() + b];
    for (uint32_t t = 0; t < count; t++) {
        SolveJob &J = *mine[t];
        const SolveDesc &d = descs[t];
        const int R = J.R, r = rank[t];
        J.X.assign((size_t)J.C * R, 0);
        for (int k = 0; k < r && k < R; k++) {
            const int c = piv[d.piv + k];
            if (c < 0 || c >= J.C) { err = "engine_solve: pivot column out of range"; return ZETA_ERR_INTERNAL; }
            std::memcpy(&J.X[(size_t)c * R], &out[d.out + (size_t)k * R], sizeof(uint64_t) * R);
        }
        J.ok = r == R;
        J.done = true;
    }
    return ZETA_OK;
}

// Whole-GPU executor (zeta_large.cuh): the host walks the plan and launches, on the engine's stream, per entry
// the formation of W (arrival block, start terms), per chunk the generation of A and M(k-1) and one step kernel
// per step (per group of eight columns), and the merge or the numerators.  Fills X.H; ms_device = the plan's
// time between CUDA events on the stream.
template <typename T, bool NARROW>
static zeta_status run_large_impl(DeviceEngine *e, LgSlot &slot, Instance &X, std::string &err, double *ms_device,
                                  uint64_t *launches) {
    if (ms_device) *ms_device = 0;
    if (launches) *launches = 0;
    uint64_t nl = 0;
    CUDA_TRY(cudaSetDevice(e->device));
    const int s = (int)X.s, b = (int)X.b, nv = (int)X.nv;
    if (NARROW && (uint64_t)X.sec_rows * X.sec_cols >= ((uint64_t)1 << 32)) {
        err = "whole-GPU executor: section of 2^32 words or more";
        return ZETA_ERR_UNSUPPORTED;
    }
    if (s < 1 || s > 4096 || b < 1 || b > 64 || X.q >= ((uint64_t)1 << 56) || X.sec.empty()) {
        err = "whole-GPU executor: needs s <= 4096, b <= 64, q < 2^56";
        return ZETA_ERR_UNSUPPORTED;
    }
    zeta_status st = upload_binom(e, err);
    if (st) return st;
    const ModQ Q = make_modq(X.q);
    // Sec R mod q (Sec R^2 mod q for the narrow path, whose generation ends with one REDC)
    std::vector<T> secR(X.sec.size());
    {
        const u128 Rm = ((u128)1 << 64) % X.q;
        const u128 Rk = NARROW ? Rm * Rm % X.q : Rm;
        for (size_t t = 0; t < X.sec.size(); t++) secR[t] = (T)((u128)X.sec[t] * Rk % X.q);
    }
    T *d_sec, *d_M, *d_A;
    uint64_t *d_W, *d_V, *d_H, *d_blocks;
    int32_t *d_monoS, *d_secrow, *d_colidx;
    Term *d_terms;
    if ((st = upload_in(slot, "lg_sec", secR, &d_sec, err))) return st;
    std::vector<T>().swap(secR);
    if ((st = upload_in(slot, "lg_monoS", X.tab_monoS, &d_monoS, err))) return st;
    if ((st = upload_in(slot, "lg_secrow", X.tab_secrow, &d_secrow, err))) return st;
    if ((st = upload_in(slot, "lg_terms", X.terms, &d_terms, err))) return st;
    const int sp = NARROW ? (s + 3) & ~3 : s;  // row stride of M and A, column stride of W and V
    const size_t ss = (size_t)s * sp, block_words = (size_t)s * b;
    const size_t cap = std::max<size_t>(X.plan.cap, 1);
    if ((st = ensure_in(slot.bufs, "lg_M", sizeof(T) * ss, (void **)&d_M, err))) return st;
    if ((st = ensure_in(slot.bufs, "lg_A", sizeof(T) * ss, (void **)&d_A, err))) return st;
    if ((st = ensure_in(slot.bufs, "lg_colidx", sizeof(int32_t) * s, (void **)&d_colidx, err))) return st;
    if ((st = ensure_in(slot.bufs, "lg_W", sizeof(uint64_t) * sp * b, (void **)&d_W, err))) return st;
    if ((st = ensure_in(slot.bufs, "lg_V", sizeof(uint64_t) * sp * b, (void **)&d_V, err))) return st;
    if ((st = ensure_in(slot.bufs, "lg_H", sizeof(uint64_t) * X.h_rows * b, (void **)&d_H, err))) return st;
    if ((st = ensure_in(slot.bufs, "lg_blocks", sizeof(uint64_t) * 2 * cap * block_words, (void **)&d_blocks, err))) return st;
    cudaStream_t stream = slot.stream;
    CUDA_TRY(cudaMemsetAsync(d_H, 0, sizeof(uint64_t) * X.h_rows * b, stream));
    CUDA_TRY(cudaMemsetAsync(d_W, 0, sizeof(uint64_t) * sp * b, stream));  // the padding rows stay zero
    CUDA_TRY(cudaMemsetAsync(d_V, 0, sizeof(uint64_t) * sp * b, stream));
    std::vector<uint64_t> tR(64, 0);  // t R mod q, the step index within a chunk in Montgomery form
    for (int t = 0; t < 64; t++) tR[t] = (uint64_t)(((u128)t << 64) % X.q);
    cudaEvent_t ev[2];
    CUDA_TRY(cudaEventCreate(&ev[0]));
    CUDA_TRY(cudaEventCreate(&ev[1]));
    CUDA_TRY(cudaEventRecord(ev[0], stream));
    auto blocks_for = [](size_t n, int t) { return (unsigned)((n + t - 1) / t); };
    const unsigned step_grid = blocks_for((size_t)s, NARROW ? kLgWarps / kLgSplit : kLgWarps);
    const int hdeg = (int)(X.d * X.n - X.n - 1);
    const Plan &P = X.plan;
    cudaError_t le = cudaSuccess;
    for (size_t ph = 0; ph + 1 < P.phase_begin.size() && le == cudaSuccess; ph++) {
        uint64_t *cur = d_blocks + (ph & 1 ? cap * block_words : 0);
        uint64_t *nxt = d_blocks + (ph & 1 ? 0 : cap * block_words);
        for (uint32_t ei = P.phase_begin[ph]; ei < P.phase_begin[ph + 1] && le == cudaSuccess; ei++) {
            const PlanEntry &E = P.entries[ei];
            LgCols cm;
            for (int t = 0; t < 64; t++) cm.col[t] = cm.lc[t] = -1;
            cm.c = 0;
            for (int col = 0; col < b; col++)
                if (E.live >> col & 1ull) {
                    cm.lc[col] = cm.c;
                    cm.col[cm.c++] = col;
                }
            if ((E.arrival >= 0 && (size_t)E.arrival >= cap) || (E.dest >= 0 && (size_t)E.dest >= cap) ||
                (E.start_chain >= 0 && (size_t)E.start_chain >= X.chains.size())) {
                err = "whole-GPU executor: plan entry out of range";
                le = cudaErrorInvalidValue;
                break;
            }
            if (cm.c == 0) {  // nothing carried: only a first contribution's clearing of its block remains
                if (E.dest >= 0 && (E.flags & 1u))
                    le = cudaMemsetAsync(nxt + (size_t)E.dest * block_words, 0, sizeof(uint64_t) * block_words, stream);
                continue;
            }
            nl++;
            k_lg_form<<<blocks_for((size_t)cm.c * s, 256), 256, 0, stream>>>(
                s, sp, b, cm, E.arrival >= 0 ? cur + (size_t)E.arrival * block_words : nullptr, d_W);
            if (E.start_chain >= 0) {
                const Chain &C = X.chains[E.start_chain];
                if (C.term_end > C.term_begin && ++nl)
                    k_lg_terms<<<blocks_for(C.term_end - C.term_begin, 256), 256, 0, stream>>>(
                        sp, cm, d_terms, C.term_begin, C.term_end, d_W, X.q);
            }
            LgVec U;
            for (int t = 0; t < kMaxVars; t++) U.x[t] = t < nv ? E.U[t] : 0;
            uint64_t *W = d_W, *V = d_V;
            for (uint32_t ci = E.chunk_begin; ci < E.chunk_end; ci++) {
                const PlanChunk &CH = P.chunks[ci];
                LgVec v;
                for (int t = 0; t < kMaxVars; t++) v.x[t] = t < nv ? CH.v[t] : 0;
                nl += 2;
                k_lg_colidx<<<blocks_for((size_t)s, 256), 256, 0, stream>>>(s, nv, (int)X.kappa, d_monoS, v, d_colidx);
                if constexpr (NARROW)
                    k_lg_gen_narrow<<<dim3(blocks_for((size_t)sp, 256), (unsigned)s), 256, 0, stream>>>(
                        s, sp, nv, X.sec_cols, d_monoS, d_secrow, d_colidx, (const uint32_t *)d_sec, U, v, Q,
                        (uint32_t *)d_M, (uint32_t *)d_A);
                else
                    k_lg_gen<T><<<blocks_for(ss, 256), 256, 0, stream>>>(s, nv, X.sec_cols, d_monoS, d_secrow, d_colidx,
                                                                         d_sec, U, v, Q, d_M, d_A);
                if (NARROW && CH.k > 64) {
                    err = "whole-GPU executor: chunk longer than 64 steps";
                    le = cudaErrorInvalidValue;
                    break;
                }
                for (int y = 0; y < CH.k; y++) {
                    for (int c0 = 0; c0 < cm.c; c0 += kLgMaxCpt) {
                        const int cg = std::min(kLgMaxCpt, cm.c - c0);
                        const uint64_t *Wg = W + (size_t)c0 * sp;
                        uint64_t *Vg = V + (size_t)c0 * sp;
                        nl++;
                        if constexpr (NARROW) {
                            // chunks with one or two columns: M(k-1) - tA on the fly; wider ones: M <- M - A
                            uint32_t *Mn = (uint32_t *)d_M;
                            const uint32_t *An = (const uint32_t *)d_A;
                            const uint64_t t = tR[y];
                            const int last = c0 + kLgMaxCpt >= cm.c;
                            if (cm.c <= 2) {
                                if (cg == 1) k_lg_step_narrow<1, false><<<step_grid, kLgWarps * 32, 0, stream>>>(s, sp, cg, Wg, Vg, Mn, An, Q, t, 0);
                                else k_lg_step_narrow<2, false><<<step_grid, kLgWarps * 32, 0, stream>>>(s, sp, cg, Wg, Vg, Mn, An, Q, t, 0);
                            } else if (cg <= 4) {
                                k_lg_step_narrow<4, true><<<step_grid, kLgWarps * 32, 0, stream>>>(s, sp, cg, Wg, Vg, Mn, An, Q, 0, last);
                            } else {
                                k_lg_step_narrow<8, true><<<step_grid, kLgWarps * 32, 0, stream>>>(s, sp, cg, Wg, Vg, Mn, An, Q, 0, last);
                            }
                        } else {
                            const int last = c0 + kLgMaxCpt >= cm.c;
                            if (cg == 1) k_lg_step<1, T><<<step_grid, kLgWarps * 32, 0, stream>>>(s, cg, Wg, Vg, d_M, d_A, Q, last);
                            else if (cg == 2) k_lg_step<2, T><<<step_grid, kLgWarps * 32, 0, stream>>>(s, cg, Wg, Vg, d_M, d_A, Q, last);
                            else if (cg <= 4) k_lg_step<4, T><<<step_grid, kLgWarps * 32, 0, stream>>>(s, cg, Wg, Vg, d_M, d_A, Q, last);
                            else k_lg_step<8, T><<<step_grid, kLgWarps * 32, 0, stream>>>(s, cg, Wg, Vg, d_M, d_A, Q, last);
                        }
                    }
                    std::swap(W, V);
                }
                for (int t = 0; t < nv; t++) U.x[t] -= CH.k * CH.v[t];
            }
            if (le != cudaSuccess) break;
            nl++;
            if (E.dest < 0)
                k_lg_numer<<<blocks_for((size_t)cm.c * s, 256), 256, 0, stream>>>(s, sp, b, nv, hdeg, U, d_monoS, cm, W, d_H,
                                                                                 X.q);
            else
                k_lg_merge<<<blocks_for(block_words, 256), 256, 0, stream>>>(s, sp, b, cm, W, nxt + (size_t)E.dest * block_words,
                                                                            (int)(E.flags & 1u), X.q);
            le = cudaGetLastError();
        }
    }
    if (le == cudaSuccess) le = cudaEventRecord(ev[1], stream);
    X.H.assign((size_t)X.h_rows * b, 0);
    if (le == cudaSuccess)
        le = cudaMemcpyAsync(X.H.data(), d_H, sizeof(uint64_t) * X.H.size(), cudaMemcpyDeviceToHost, stream);
    if (le == cudaSuccess) le = cudaStreamSynchronize(stream);
    float ms = 0;
    if (le == cudaSuccess) cudaEventElapsedTime(&ms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (le == cudaErrorInvalidValue && !err.empty()) return ZETA_ERR_INTERNAL;
    CUDA_TRY(le);
    if (ms_device) *ms_device = ms;
    if (launches) *launches = nl;
    X.steps = P.steps;
    X.column_steps = P.column_steps;
    X.chunks = P.chunks_played;
    return ZETA_OK;
}

static zeta_status run_large_on(DeviceEngine *e, LgSlot &slot, Instance &X, std::string &err, double *ms_device,
                                uint64_t *launches) {
    if (X.q < ((uint64_t)1 << 26)) return run_large_impl<uint32_t, true>(e, slot, X, err, ms_device, launches);
    return X.q < ((uint64_t)1 << 32) ? run_large_impl<uint32_t, false>(e, slot, X, err, ms_device, launches)
                                     : run_large_impl<uint64_t, false>(e, slot, X, err, ms_device, launches);
}

// Lanes 0 .. n-1 of the whole-GPU executor (lane 0 on the engine's stream, the others on streams of their own).
static zeta_status lg_lanes(DeviceEngine *e, size_t n, std::string &err) {
    if (e->lg.empty()) {
        e->lg.emplace_back();
        e->lg[0].stream = e->stream;
    }
    while (e->lg.size() < n) {
        LgSlot sl;
        CUDA_TRY(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
        sl.owned = true;
        e->lg.push_back(std::move(sl));
    }
    return ZETA_OK;
}

constexpr size_t kLgLanes = 8;

static double steady_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

zeta_status engine_run_large(DeviceEngine *e, std::vector<Instance *> &xs, std::string &err, double *ms_device,
                             uint64_t *launches, double t_ref_ms) {
    *ms_device = 0;
    *launches = 0;
    if (xs.empty()) return ZETA_OK;
    CUDA_TRY(cudaSetDevice(e->device));
    zeta_status st = upload_binom(e, err);
    if (st) return st;
    if ((st = lg_lanes(e, 1, err))) return st;
    std::vector<Instance *> whole, shared;
    for (Instance *X : xs) (X->s > 512 ? whole : shared).push_back(X);
    // smaller ones first (quintic surfaces: s = 455, about 10 000 short launches each), so that a stream's short
    // instances do not wait for its cubic fourfold; they leave most SMs idle and are bound by launch latency: up to
    // eight at a time, each lane driven by a host thread of its own
    const size_t G = std::min(kLgLanes, shared.size());  // 0: no thread
    if ((st = lg_lanes(e, std::max<size_t>(G, 1), err))) return st;
    std::vector<zeta_status> sts(G, ZETA_OK);
    std::vector<std::string> errs(G);
    std::vector<uint64_t> nls(G, 0);
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<std::thread> pool;
    for (size_t g = 0; g < G; g++)
        pool.emplace_back([&, g]() {
            if (cudaSetDevice(e->device) != cudaSuccess) {
                sts[g] = ZETA_ERR_DEVICE;
                errs[g] = "cudaSetDevice";
                return;
            }
            for (size_t i = g; i < shared.size(); i += G) {
                double ms = 0;
                uint64_t nl = 0;
                shared[i]->ms_dev_start = steady_ms() - t_ref_ms;
                const zeta_status s2 = run_large_on(e, e->lg[g], *shared[i], errs[g], &ms, &nl);
                shared[i]->ms_dev_end = steady_ms() - t_ref_ms;
                if (s2) {
                    sts[g] = s2;
                    return;
                }
                nls[g] += nl;
            }
        });
    for (auto &t : pool) t.join();
    for (size_t g = 0; g < G; g++)
        if (sts[g]) {
            err = errs[g];
            return sts[g];
        }
    if (!shared.empty())
        *ms_device += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (uint64_t nl : nls) *launches += nl;
    // then the instances with s > 512, which fill the GPU: one at a time on lane 0
    for (Instance *X : whole) {
        double ms = 0;
        uint64_t nl = 0;
        X->ms_dev_start = steady_ms() - t_ref_ms;
        if ((st = run_large_on(e, e->lg[0], *X, err, &ms, &nl))) return st;
        X->ms_dev_end = steady_ms() - t_ref_ms;
        *ms_device += ms;
        *launches += nl;
    }
    return ZETA_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the kernel-level entry point (zeta_horner_static).
// Its matrix scratch lives in this file-scope device array; every call on a
// device shares it.  The last 32 words hold the call's status flag.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchWords = (size_t)2 << 20;  // 2 Mi uint64 = 16 MiB per device
constexpr size_t kStaticStatusWord = kStaticScratchWords - 32;
static __device__ __align__(256) uint64_t g_static_scratch[kStaticScratchWords];

// ModQ of q computed on the device (no host round trip): -q^{-1} mod 2^64 by
// Newton iteration, 2^64 mod q as (2^64 - q) mod q, then modular doublings.
__device__ ModQ modq_on_device(uint64_t q) {
    ModQ Q;
    Q.q = q;
    uint64_t inv = 1;
    for (int i = 0; i < 7; i++) inv *= 2 - q * inv;
    Q.qneg_inv = (uint64_t)0 - inv;
    const uint64_t r = ((uint64_t)0 - q) % q;  // 2^64 mod q
    uint64_t r2 = r, k30 = r;
    for (int i = 0; i < 64; i++) { r2 <<= 1; if (r2 >= q) r2 -= q; }   // 2^128 mod q
    for (int i = 0; i < 30; i++) { k30 <<= 1; if (k30 >= q) k30 -= q; } // 2^30 2^64 mod q
    Q.r2 = r2;
    Q.k30 = k30;
    return Q;
}

template <int CPT>
__global__ void __launch_bounds__(512) k_horner_problems_static(
    uint32_t count, int s, int c, const uint32_t *__restrict__ kk, const uint64_t *__restrict__ A,
    const uint64_t *__restrict__ B, uint64_t *__restrict__ W, const uint64_t *__restrict__ qv,
    uint64_t *__restrict__ scratch) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t MASK30 = (1u << 30) - 1;
    uint64_t *Ms = scratch + (size_t)blockIdx.x * 2 * s * s;
    uint64_t *As = Ms + (size_t)s * s;
    uint2 *Wl = (uint2 *)smem_raw;
    uint2 *Vl = Wl + (size_t)s * pad4(c);
    const int cs = pad4(c);
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        const uint64_t q = qv[t];
        if (q < 3 || q > ((uint64_t)1 << 60) || !(q & 1) || (uint64_t)s >= 8 * q) {
            if (threadIdx.x == 0) atomicOr((unsigned long long *)&scratch[kStaticStatusWord], 1ull);
            continue;  // uniform across the block: W_t is left unchanged
        }
        const ModQ Q = modq_on_device(q);
        const int k = (int)kk[t];
        const uint64_t *At_g = A + (size_t)t * s * s;
        const uint64_t *Bt_g = B + (size_t)t * s * s;
        uint64_t *Wt = W + (size_t)t * s * c;
        for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
            const int r = e / s, j = e % s;  // row-major input
            const uint64_t a = to_mont(At_g[e], Q), b = to_mont(Bt_g[e], Q);
            As[(size_t)j * s + r] = a;
            Ms[(size_t)j * s + r] = addmod(mul_small(a, (uint64_t)(k > 0 ? k - 1 : 0), Q), b, Q.q);
        }
        for (int e = threadIdx.x; e < s * cs; e += blockDim.x) {
            const int j = e / cs, col = e - j * cs;
            const uint64_t w = col < c ? Wt[j * c + col] : 0;
            Wl[e] = make_uint2((uint32_t)w & MASK30, (uint32_t)(w >> 30));
        }
        __syncthreads();
        const int res = horner_block<CPT>(s, c, k, Ms, As, Wl, Vl, Q);
        const uint2 *R = res ? Vl : Wl;
        for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
            const int j = e / c, col = e - j * c;
            Wt[e] = ((uint64_t)R[j * cs + col].y << 30) | R[j * cs + col].x;
        }
        __syncthreads();
    }
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
uint64_t *g_static_ptr[kMaxDevices];  // cached only after a successful lookup
}  // namespace

// Device address of g_static_scratch on the current device.  The lookup runs
// on the first call on a device and is cached only when it succeeds, so a
// failed first call (for example one made during a stream capture) is
// retried by the next call.
static cudaError_t static_scratch(int dev, uint64_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        uint64_t *ptr = nullptr;
        const cudaError_t ce = cudaGetSymbolAddress((void **)&ptr, g_static_scratch);
        if (ce != cudaSuccess || !ptr) {
            cudaGetLastError();
            return ce != cudaSuccess ? ce : cudaErrorInvalidSymbol;
        }
        g_static_ptr[dev] = ptr;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

}  // namespace zeta

extern "C" zeta_status zeta_horner_static(void *cuda_stream, uint32_t count, uint32_t s, uint32_t c,
                                          const uint32_t *k, const uint64_t *A, const uint64_t *B, uint64_t *W,
                                          const uint64_t *q) {
    using namespace zeta;
    if (count && (!k || !A || !B || !W || !q)) return ZETA_ERR_ARG;
    if (s == 0 || c == 0 || s > (uint32_t)kMaxS || c > (uint32_t)kMaxC) return ZETA_ERR_ARG;
    const size_t per_block = (size_t)2 * s * s;
    if (per_block > kStaticStatusWord) return ZETA_ERR_ARG;
    const size_t smem = (size_t)2 * s * pad4((int)c) * sizeof(uint2);
    if (smem > 227 * 1024) return ZETA_ERR_ARG;
    if (count == 0) return ZETA_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return ZETA_ERR_DEVICE; }
    uint64_t *scratch = nullptr;
    if (static_scratch(dev, &scratch) != cudaSuccess || !scratch) { cudaGetLastError(); return ZETA_ERR_DEVICE; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ZETA_ERR_DEVICE;
    const size_t fit = kStaticStatusWord / per_block;
    const int grid = (int)std::min<size_t>(std::min<size_t>(count, fit), (size_t)sms * 4);
    const int threads = launch_threads((int)s, (int)c);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaFuncSetAttribute((const void *)k_horner_problems_static<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) { cudaGetLastError(); return ZETA_ERR_DEVICE; }
    // the status word must start at zero for every call
    if (cudaMemsetAsync(scratch + kStaticStatusWord, 0, sizeof(uint64_t), st) != cudaSuccess) return ZETA_ERR_DEVICE;
    k_horner_problems_static<4><<<grid, threads, smem, st>>>(count, (int)s, (int)c, k, A, B, W, q, scratch);
    if (cudaGetLastError() != cudaSuccess) return ZETA_ERR_DEVICE;
    uint64_t flag = 0;
    if (cudaMemcpyAsync(&flag, scratch + kStaticStatusWord, sizeof(flag), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ZETA_ERR_DEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ZETA_ERR_DEVICE;
    return flag ? ZETA_ERR_ARG : ZETA_OK;
}

