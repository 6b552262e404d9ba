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
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
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

constexpr int kThreads = 256;
constexpr int kMaxS = 512;
constexpr int kMaxC = 32;

// ---------------------------------------------------------------------------
// Modular arithmetic on the device
// ---------------------------------------------------------------------------
struct ModQ {
    uint64_t q;
    uint64_t qneg_inv;  // -q^{-1} mod 2^64
    uint64_t r2;        // 2^128 mod q
    uint64_t k[3];      // 2^128 * 2^{30 t} mod q, t = 0, 1, 2
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

// out = T0 + T1 2^30 + T2 2^60 mod q, each T_t a 128-bit value below q 2^64.
__device__ __forceinline__ uint64_t fold_limbs(const uint64_t T[6], const ModQ &Q) {
    uint64_t out = 0;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        uint64_t y = redc(T[2 * t], T[2 * t + 1], Q);  // T_t 2^{-64}
        uint64_t z = redc(y * Q.k[t], mul_hi64(y, Q.k[t]), Q);  // T_t 2^{30t} mod q
        out = addmod(out, z, Q.q);
    }
    return out;
}

// ---------------------------------------------------------------------------
// One block-wide evaluation of k steps of Algorithm 2.
//  Mt, At: s x s stored transposed (entry (row r, col j) at [j*s + r]); Mt
//          holds M(k-1) = (k-1)A + B on entry and is consumed.
//  W0/W1 : shared memory limbs (low 30 bits / high bits) of W, s x c, [j*c + col];
//  V0/V1 : second buffer of the same shape.  On return the result is in the
//          buffer returned (0 = W, 1 = V).
// ---------------------------------------------------------------------------
template <int CPT>
__device__ int horner_block(int s, int c, int k, uint64_t *Mt, const uint64_t *At,
                            uint32_t *W0, uint32_t *W1, uint32_t *V0, uint32_t *V1, const ModQ &Q) {
    const int ngroups = (c + CPT - 1) / CPT;
    const int items = s * ngroups;
    const uint32_t MASK = (1u << 30) - 1;
    int cur = 0;
    for (int step = 0; step < k; step++) {
        uint32_t *in0 = cur ? V0 : W0, *in1 = cur ? V1 : W1;
        uint32_t *out0 = cur ? W0 : V0, *out1 = cur ? W1 : V1;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int r = it % s;
            const int g = it / s;
            const int c0 = g * CPT;
            uint64_t T[CPT][6];
#pragma unroll
            for (int cc = 0; cc < CPT; cc++)
#pragma unroll
                for (int t = 0; t < 6; t++) T[cc][t] = 0;
            for (int jb = 0; jb < s; jb += 4) {
                uint64_t S[CPT][3];
#pragma unroll
                for (int cc = 0; cc < CPT; cc++) S[cc][0] = S[cc][1] = S[cc][2] = 0;
                const int jend = min(jb + 4, s);
                for (int j = jb; j < jend; j++) {
                    const uint64_t m = Mt[(size_t)j * s + r];
                    const uint32_t m0 = (uint32_t)m & MASK;
                    const uint32_t m1 = (uint32_t)(m >> 30);
#pragma unroll
                    for (int cc = 0; cc < CPT; cc++) {
                        const int col = c0 + cc;
                        if (col < c) {
                            const uint32_t w0 = in0[j * c + col];
                            const uint32_t w1 = in1[j * c + col];
                            S[cc][0] += (uint64_t)m0 * w0;
                            S[cc][1] += (uint64_t)m0 * w1 + (uint64_t)m1 * w0;
                            S[cc][2] += (uint64_t)m1 * w1;
                        }
                    }
                }
#pragma unroll
                for (int cc = 0; cc < CPT; cc++) {
                    add128(T[cc][0], T[cc][1], S[cc][0]);
                    add128(T[cc][2], T[cc][3], S[cc][1]);
                    add128(T[cc][4], T[cc][5], S[cc][2]);
                }
            }
#pragma unroll
            for (int cc = 0; cc < CPT; cc++) {
                const int col = c0 + cc;
                if (col < c) {
                    uint64_t v = fold_limbs(T[cc], Q);
                    out0[r * c + col] = (uint32_t)v & MASK;
                    out1[r * c + col] = (uint32_t)(v >> 30);
                }
            }
        }
        __syncthreads();
        if (step + 1 < k) {
            for (int e = threadIdx.x; e < s * s; e += blockDim.x) Mt[e] = submod(Mt[e], At[e], Q.q);
            __syncthreads();
        }
        cur ^= 1;
    }
    return cur;
}

// ---------------------------------------------------------------------------
// Device data of a batch
// ---------------------------------------------------------------------------
struct DInst {
    ModQ Q;
    uint32_t n, d, b, s, nv;
    uint32_t sec_cols, h_rows, kappa;
    uint32_t tab;          // table set index
    uint64_t sec_off;      // into sec pool
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

struct DItem {
    uint32_t inst;
    uint32_t chain_begin, chain_end;
    uint32_t slot;         // partial H slot
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

// Algorithm 3 (greedy v) with S = {0..n}, and the largest chunk of Sec. 4.2.
__device__ void greedy_chunk(const int *U, int nv, int n, int d, int *v, int *k_out) {
    int i = d;
    for (int t = 0; t < nv; t++) v[t] = 0;
    for (int t = 0; t < nv && i > 0; t++)
        if (U[t] != 0) { v[t] = 1; i--; }
    while (i > 0) {
        for (int t = 0; t < nv && i > 0; t++)
            if (v[t] < U[t]) { v[t]++; i--; }
    }
    int norm = 0;
    for (int t = 0; t < nv; t++) norm += U[t];
    int k = (norm - n) / d;
    for (int t = 0; t < nv; t++)
        if (v[t] > 0) k = min(k, U[t] / v[t]);
    *k_out = k;
}

// Shared-memory layout of the chain kernel (bytes)
__host__ __device__ inline size_t chain_smem(int s, int c, int h_rows) {
    return (size_t)4 * s * c * sizeof(uint32_t) + (size_t)h_rows * c * sizeof(uint64_t) + (size_t)s * sizeof(int) + 64;
}

// Persistent kernel: each block takes work items (ranges of chains of one
// instance) from a queue and plays the depth-first policy (Sec. 4.2) on
// each chain to pole order n, accumulating x^U g / x^S into H.
template <int CPT>
__global__ void __launch_bounds__(kThreads) k_depth_first(
    const DInst *__restrict__ insts, const DTab *__restrict__ tabs, const int32_t *__restrict__ tabpool,
    const uint64_t *__restrict__ secpool, const DChain *__restrict__ chains, const Term *__restrict__ terms,
    const DItem *__restrict__ items, uint32_t nitems, uint32_t *__restrict__ queue,
    uint64_t *__restrict__ scratch, size_t scratch_stride, uint64_t *__restrict__ partial,
    size_t partial_stride, unsigned long long *__restrict__ counters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int sU[kMaxVars], sv[kMaxVars], sx[kMaxVars], sk;
    __shared__ uint32_t s_item;
    uint64_t *Mt = scratch + (size_t)blockIdx.x * scratch_stride;
    unsigned long long my_chunks = 0, my_steps = 0;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t itx = s_item;
        __syncthreads();
        if (itx >= nitems) break;
        const DItem item = items[itx];
        const DInst I = insts[item.inst];
        const DTab T = tabs[I.tab];
        const int s = (int)I.s, c = (int)I.b, nv = (int)I.nv, n = (int)I.n, d = (int)I.d;
        const int32_t *monoS = tabpool + T.monoS_off;
        const int32_t *secrow = tabpool + T.secrow_off;
        const uint64_t *Sec = secpool + I.sec_off;
        uint64_t *At = Mt + (size_t)s * s;
        uint32_t *W0 = (uint32_t *)smem_raw;
        uint32_t *W1 = W0 + s * c;
        uint32_t *V0 = W1 + s * c;
        uint32_t *V1 = V0 + s * c;
        uint64_t *Hs = (uint64_t *)(V1 + s * c);
        int *colidx = (int *)(Hs + (size_t)I.h_rows * c);
        const uint32_t MASK = (1u << 30) - 1;
        for (int e = threadIdx.x; e < (int)I.h_rows * c; e += blockDim.x) Hs[e] = 0;
        for (uint32_t ch = item.chain_begin; ch < item.chain_end; ch++) {
            const DChain C = chains[ch];
            for (int e = threadIdx.x; e < s * c; e += blockDim.x) { W0[e] = 0; W1[e] = 0; }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (uint32_t t = C.term_begin; t < C.term_end; t++) {
                    const Term tm = terms[t];
                    const int e = (int)tm.row * c + (int)tm.col;
                    uint64_t old = ((uint64_t)W1[e] << 30) | W0[e];
                    uint64_t nw = addmod(old, tm.coeff, I.Q.q);
                    W0[e] = (uint32_t)nw & MASK;
                    W1[e] = (uint32_t)(nw >> 30);
                }
                for (int t = 0; t < nv; t++) sU[t] = C.U[t];
            }
            __syncthreads();
            int cur = 0;  // 0: data in W, 1: data in V
            while (true) {
                if (threadIdx.x == 0) {
                    int norm = 0;
                    for (int t = 0; t < nv; t++) norm += sU[t];
                    if (norm > n) {
                        int v[kMaxVars], k;
                        greedy_chunk(sU, nv, n, d, v, &k);
                        for (int t = 0; t < nv; t++) { sv[t] = v[t]; sx[t] = sU[t] - k * v[t]; }
                        sk = k;
                    } else {
                        sk = 0;
                    }
                }
                __syncthreads();
                const int k = sk;
                if (k == 0) break;
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
                // A and M(k-1) = (k-1) A + B from the section
                for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
                    const int r = e % s, j = e / s;
                    const int col = colidx[j];
                    uint64_t aL = 0, aH = 0, bL = 0, bH = 0;
                    if (col >= 0) {
                        for (int i = 0; i < nv; i++) {
                            const int row = secrow[i * s + r];
                            if (row < 0) continue;
                            const uint64_t val = __ldg(&Sec[(size_t)row * I.sec_cols + col]);
                            const uint64_t wa = (uint64_t)sv[i];
                            const uint64_t wb = (uint64_t)(sx[i] + monoS[r * nv + i]);
                            add128(aL, aH, val * wa);
                            aH += mul_hi64(val, wa);
                            add128(bL, bH, val * wb);
                            bH += mul_hi64(val, wb);
                        }
                    }
                    const uint64_t A = reduce128(aL, aH, I.Q);
                    const uint64_t B = reduce128(bL, bH, I.Q);
                    At[(size_t)j * s + r] = A;
                    Mt[(size_t)j * s + r] = addmod(mul_small(A, (uint64_t)(k - 1), I.Q), B, I.Q.q);
                }
                __syncthreads();
                int res;
                if (cur == 0) res = horner_block<CPT>(s, c, k, Mt, At, W0, W1, V0, V1, I.Q);
                else res = horner_block<CPT>(s, c, k, Mt, At, V0, V1, W0, W1, I.Q);
                cur ^= res;
                if (threadIdx.x == 0) {
                    for (int t = 0; t < nv; t++) sU[t] = sx[t];
                    my_chunks++;
                    my_steps += k;
                }
                __syncthreads();
            }
            // accumulate x^U g / x^S (pole order n) into H
            const uint32_t *R0 = cur ? V0 : W0, *R1 = cur ? V1 : W1;
            const int hdeg = d * n - n - 1;
            for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
                const int j = e / c, col = e % c;
                uint64_t val = ((uint64_t)R1[e] << 30) | R0[e];
                if (!val) continue;
                int g[kMaxVars];
                bool ok = true;
                for (int t = 0; t < nv; t++) {
                    g[t] = sU[t] + monoS[j * nv + t] - 1;
                    if (g[t] < 0) ok = false;
                }
                if (!ok) continue;  // cannot carry a coefficient on a valid path
                const int h = dev_rank(g, nv, hdeg);
                Hs[h * c + col] = addmod(Hs[h * c + col], val, I.Q.q);
            }
            __syncthreads();
        }
        uint64_t *out = partial + (size_t)item.slot * partial_stride;
        for (int e = threadIdx.x; e < (int)I.h_rows * c; e += blockDim.x) out[e] = Hs[e];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&counters[0], my_chunks);
        atomicAdd(&counters[1], my_steps);
    }
}

// H of each instance = sum of its items' partial slots mod q.
__global__ void k_sum_partials(const DInst *__restrict__ insts, const uint32_t *__restrict__ slot_begin,
                               const uint32_t *__restrict__ slot_end, const uint64_t *__restrict__ partial,
                               size_t partial_stride, uint64_t *__restrict__ H, size_t h_stride, uint32_t ninst) {
    const uint32_t i = blockIdx.x;
    if (i >= ninst) return;
    const DInst I = insts[i];
    const int len = (int)(I.h_rows * I.b);
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        uint64_t acc = 0;
        for (uint32_t sl = slot_begin[i]; sl < slot_end[i]; sl++)
            acc = addmod(acc, partial[(size_t)sl * partial_stride + e], I.Q.q);
        H[(size_t)i * h_stride + e] = acc;
    }
}

// Kernel-level Algorithm 2 on independent problems (zeta_horner_device).
template <int CPT>
__global__ void __launch_bounds__(kThreads) k_horner_problems(
    uint32_t count, int s, int c, const uint32_t *__restrict__ kk, const uint64_t *__restrict__ A,
    const uint64_t *__restrict__ B, uint64_t *__restrict__ W, const ModQ *__restrict__ mods,
    uint64_t *__restrict__ scratch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t MASK = (1u << 30) - 1;
    uint64_t *Mt = scratch + (size_t)blockIdx.x * 2 * s * s;
    uint64_t *At = Mt + (size_t)s * s;
    uint32_t *W0 = (uint32_t *)smem_raw;
    uint32_t *W1 = W0 + s * c;
    uint32_t *V0 = W1 + s * c;
    uint32_t *V1 = V0 + s * c;
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        const ModQ Q = mods[t];
        const int k = (int)kk[t];
        const uint64_t *At_g = A + (size_t)t * s * s;
        const uint64_t *Bt_g = B + (size_t)t * s * s;
        uint64_t *Wt = W + (size_t)t * s * c;
        for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
            const int r = e / s, j = e % s;  // row-major input
            const uint64_t a = At_g[e], b = Bt_g[e];
            At[(size_t)j * s + r] = a;
            Mt[(size_t)j * s + r] = addmod(mul_small(a, (uint64_t)(k > 0 ? k - 1 : 0), Q), b, Q.q);
        }
        for (int e = threadIdx.x; e < s * c; e += blockDim.x) {
            const uint64_t w = Wt[e];
            W0[e] = (uint32_t)w & MASK;
            W1[e] = (uint32_t)(w >> 30);
        }
        __syncthreads();
        int res = horner_block<CPT>(s, c, k, Mt, At, W0, W1, V0, V1, Q);
        const uint32_t *R0 = res ? V0 : W0, *R1 = res ? V1 : W1;
        for (int e = threadIdx.x; e < s * c; e += blockDim.x) Wt[e] = ((uint64_t)R1[e] << 30) | R0[e];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct DeviceEngine {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sms = 0;
    std::map<std::string, DevBuf> bufs;
    bool binom_ready = false;
};

static zeta_status ensure(DeviceEngine *e, const char *name, size_t bytes, void **out, std::string &err) {
    DevBuf &b = e->bufs[name];
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

static ModQ make_modq(uint64_t q) {
    ModQ Q;
    Q.q = q;
    uint64_t inv = 1;
    for (int i = 0; i < 7; i++) inv *= 2 - q * inv;
    Q.qneg_inv = (uint64_t)0 - inv;
    u128 R = ((u128)1 << 64) % q;
    Q.r2 = (uint64_t)(R * R % q);
    for (int t = 0; t < 3; t++) Q.k[t] = (uint64_t)((u128)Q.r2 * (((u128)1 << (30 * t)) % q) % q);
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

void engine_destroy(DeviceEngine *e) {
    if (!e) return;
    cudaSetDevice(e->device);
    for (auto &kv : e->bufs)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
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

static int host_rank(const int *ex, int nv, int deg) {
    long long idx = 0;
    int rem = deg;
    for (int i = 0; i < nv - 1; i++) {
        int k = nv - i - 1;
        int top = rem - ex[i] - 1;
        if (top >= 0) {
            long long r = 1;
            for (int t = 1; t <= k; t++) r = r * (top + t) / t;
            idx += r;
        }
        rem -= ex[i];
    }
    return (int)idx;
}

static void host_monos(int nv, int deg, std::vector<int> &out) {
    std::vector<int> cur(nv, 0);
    std::function<void(int, int)> rec = [&](int pos, int rem) {
        if (pos == nv - 1) {
            cur[pos] = rem;
            out.insert(out.end(), cur.begin(), cur.end());
            return;
        }
        for (int t = rem; t >= 0; t--) {
            cur[pos] = t;
            rec(pos + 1, rem - t);
        }
    };
    if (deg >= 0) rec(0, deg);
}

struct DeviceBatch {
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
    DItem *d_items = nullptr;
    uint32_t *d_sb = nullptr, *d_se = nullptr, *d_queue = nullptr;
    uint64_t *d_scratch = nullptr, *d_partial = nullptr, *d_H = nullptr;
    unsigned long long *d_counters = nullptr;
    uint32_t nitems = 0;
    int grid = 1, CPT = 4;
    size_t smem = 0, scratch_stride = 0, partial_stride = 0;
    uint64_t bytes = 0, bytes_h2d = 0, bytes_d2h = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;  // around each recurrence launch
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
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, e->stream));
    B->bytes_h2d += sizeof(T) * v.size();
    return ZETA_OK;
}

void engine_release(DeviceBatch *B) {
    if (!B) return;
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
                           DeviceBatch **out, std::string &err) {
    *out = nullptr;
    CUDA_TRY(cudaSetDevice(e->device));
    zeta_status st = upload_binom(e, err);
    if (st) return st;
    DeviceBatch *B = new (std::nothrow) DeviceBatch();
    if (!B) return ZETA_ERR_OOM;
    B->insts = batch;
    B->policy = policy;
    B->path = path;

    // tables per (n, d)
    std::map<std::pair<int, int>, uint32_t> tab_of;
    std::vector<DTab> tabs;
    std::vector<int32_t> tabpool;
    std::vector<DInst> dinst;
    std::vector<uint64_t> secpool;
    std::vector<DChain> dchains;
    std::vector<Term> dterms;
    std::vector<DItem> ditems;
    std::vector<uint32_t> slot_begin, slot_end;
    std::vector<uint64_t> item_w;
    int max_s = 0, max_c = 0, max_h = 0;
    uint64_t total_work = 0;
    for (Instance *X : batch)
        for (auto &ch : X->chains) total_work += ch.work;
    const int blocks_target = std::max(1, e->sms);
    const uint64_t item_work = std::max<uint64_t>(1, total_work / ((uint64_t)blocks_target * 8));
    for (size_t ii = 0; ii < batch.size(); ii++) {
        Instance *X = batch[ii];
        auto key = std::make_pair((int)X->n, (int)X->d);
        if (!tab_of.count(key)) {
            DTab T;
            T.nv = X->nv;
            T.s = X->s;
            T.h_rows = X->h_rows;
            std::vector<int> mS;
            host_monos(X->nv, X->d * X->n - X->n, mS);
            T.monoS_off = (uint32_t)tabpool.size();
            tabpool.insert(tabpool.end(), mS.begin(), mS.end());
            // secrow[i][omega] = row (i, omega - 1 + e_i) of Sec, -1 if a coordinate is negative
            int srcdeg = X->n * (X->d - 2);
            std::vector<int> tmp;
            host_monos(X->nv, srcdeg, tmp);
            int nsrc = (int)tmp.size() / X->nv;
            T.secrow_off = (uint32_t)tabpool.size();
            for (uint32_t i = 0; i < X->nv; i++)
                for (uint32_t r = 0; r < X->s; r++) {
                    int g[kMaxVars];
                    bool ok = true;
                    for (uint32_t t = 0; t < X->nv; t++) {
                        g[t] = mS[r * X->nv + t] - 1 + (t == i ? 1 : 0);
                        if (g[t] < 0) ok = false;
                    }
                    tabpool.push_back(ok ? (int32_t)(i * nsrc + host_rank(g, X->nv, srcdeg)) : -1);
                }
            tab_of[key] = (uint32_t)tabs.size();
            tabs.push_back(T);
        }
        DInst I;
        I.Q = make_modq(X->q);
        I.n = X->n; I.d = X->d; I.b = X->b; I.s = X->s; I.nv = X->nv;
        I.sec_cols = X->sec_cols; I.h_rows = X->h_rows; I.kappa = X->kappa;
        I.tab = tab_of[key];
        I.sec_off = secpool.size();
        secpool.insert(secpool.end(), X->sec.begin(), X->sec.end());
        dinst.push_back(I);
        max_s = std::max(max_s, (int)X->s);
        max_c = std::max(max_c, (int)X->b);
        max_h = std::max(max_h, (int)X->h_rows);
        uint32_t cbase = (uint32_t)dchains.size();
        uint32_t tbase = (uint32_t)dterms.size();
        for (auto &ch : X->chains) {
            DChain dc;
            std::memcpy(dc.U, ch.U, sizeof(dc.U));
            dc.term_begin = ch.term_begin + tbase;
            dc.term_end = ch.term_end + tbase;
            dchains.push_back(dc);
        }
        dterms.insert(dterms.end(), X->terms.begin(), X->terms.end());
        // work items: consecutive chains with about item_work each
        slot_begin.push_back((uint32_t)ditems.size());
        uint32_t start = 0;
        uint64_t acc = 0;
        for (uint32_t c = 0; c < X->chains.size(); c++) {
            acc += X->chains[c].work;
            if (acc >= item_work || c + 1 == X->chains.size()) {
                ditems.push_back(DItem{(uint32_t)ii, cbase + start, cbase + c + 1, (uint32_t)ditems.size()});
                item_w.push_back(acc);
                start = c + 1;
                acc = 0;
            }
        }
        if (X->chains.empty()) {
            ditems.push_back(DItem{(uint32_t)ii, cbase, cbase, (uint32_t)ditems.size()});
            item_w.push_back(0);
        }
        slot_end.push_back((uint32_t)ditems.size());
    }
    if (max_s > kMaxS || max_c > kMaxC) {
        err = "instance too large for the device kernels";
        engine_release(B);
        return ZETA_ERR_UNSUPPORTED;
    }
    // largest items first (longest-processing-time order for the persistent queue)
    std::stable_sort(ditems.begin(), ditems.end(), [&](const DItem &a, const DItem &b) { return item_w[a.slot] > item_w[b.slot]; });
    B->nitems = (uint32_t)ditems.size();
#define UP(vec, ptr) if ((st = dev_upload(e, B, vec, &B->ptr, err))) { engine_release(B); return st; }
    UP(dinst, d_inst);
    UP(tabs, d_tabs);
    UP(tabpool, d_tabpool);
    UP(secpool, d_sec);
    UP(dchains, d_chains);
    UP(dterms, d_terms);
    UP(ditems, d_items);
    UP(slot_begin, d_sb);
    UP(slot_end, d_se);
#undef UP
    B->smem = chain_smem(max_s, max_c, max_h);
    B->CPT = max_c <= 6 ? 2 : (max_c <= 12 ? 3 : 4);
    const void *kfn = B->CPT == 2 ? (const void *)k_depth_first<2>
                    : B->CPT == 3 ? (const void *)k_depth_first<3> : (const void *)k_depth_first<4>;
    CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, B->smem));
    per_sm = std::max(1, per_sm);
    B->grid = std::max(1, (int)std::min<size_t>((size_t)e->sms * per_sm, ditems.size()));
    B->scratch_stride = (size_t)2 * max_s * max_s;
    B->partial_stride = (size_t)max_h * max_c;
#define AL(count, ptr) if ((st = dev_alloc(B, count, &B->ptr, err))) { engine_release(B); return st; }
    AL(B->scratch_stride * B->grid, d_scratch);
    AL(B->partial_stride * ditems.size(), d_partial);
    AL(B->partial_stride * batch.size(), d_H);
    AL(16, d_queue);
    AL(8, d_counters);
#undef AL
    *out = B;
    return ZETA_OK;
}

zeta_status engine_launch(DeviceEngine *e, DeviceBatch *B, std::string &err) {
    CUDA_TRY(cudaSetDevice(e->device));
    CUDA_TRY(cudaMemsetAsync(B->d_queue, 0, 16 * sizeof(uint32_t), e->stream));
    CUDA_TRY(cudaMemsetAsync(B->d_counters, 0, 8 * sizeof(unsigned long long), e->stream));
    cudaEvent_t ev0, ev1;
    CUDA_TRY(cudaEventCreate(&ev0));
    CUDA_TRY(cudaEventCreate(&ev1));
    B->events.push_back({ev0, ev1});
    CUDA_TRY(cudaEventRecord(ev0, e->stream));
#define LAUNCH(C)                                                                                          \
    k_depth_first<C><<<B->grid, kThreads, B->smem, e->stream>>>(                                           \
        B->d_inst, B->d_tabs, B->d_tabpool, B->d_sec, B->d_chains, B->d_terms, B->d_items, B->nitems,       \
        B->d_queue, B->d_scratch, B->scratch_stride, B->d_partial, B->partial_stride, B->d_counters)
    if (B->CPT == 2) LAUNCH(2);
    else if (B->CPT == 3) LAUNCH(3);
    else LAUNCH(4);
#undef LAUNCH
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(ev1, e->stream));
    k_sum_partials<<<(unsigned)B->insts.size(), 256, 0, e->stream>>>(B->d_inst, B->d_sb, B->d_se, B->d_partial,
                                                                    B->partial_stride, B->d_H, B->partial_stride,
                                                                    (uint32_t)B->insts.size());
    CUDA_TRY(cudaGetLastError());
    return ZETA_OK;
}

zeta_status engine_collect(DeviceEngine *e, DeviceBatch *B, std::string &err) {
    CUDA_TRY(cudaSetDevice(e->device));
    std::vector<uint64_t> hH(B->partial_stride * B->insts.size());
    unsigned long long hc[8] = {0};
    CUDA_TRY(cudaMemcpyAsync(hH.data(), B->d_H, sizeof(uint64_t) * hH.size(), cudaMemcpyDeviceToHost, e->stream));
    CUDA_TRY(cudaMemcpyAsync(hc, B->d_counters, sizeof(hc), cudaMemcpyDeviceToHost, e->stream));
    CUDA_TRY(cudaStreamSynchronize(e->stream));
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
    for (size_t ii = 0; ii < B->insts.size(); ii++) {
        Instance *X = B->insts[ii];
        X->H.assign(hH.begin() + ii * B->partial_stride, hH.begin() + ii * B->partial_stride + (size_t)X->h_rows * X->b);
        X->steps = 0;
        X->column_steps = 0;
        for (auto &ch : X->chains) {
            int norm = 0;
            for (uint32_t t = 0; t < X->nv; t++) norm += ch.U[t];
            uint64_t steps = (uint64_t)(norm - (int)X->n) / X->d;
            X->steps += steps;
            std::vector<char> live(X->b, 0);
            for (uint32_t t = ch.term_begin; t < ch.term_end; t++) live[X->terms[t].col] = 1;
            uint64_t lc = 0;
            for (char l : live) lc += l;
            X->column_steps += steps * lc;
        }
        X->chunks = 0;
    }
    if (!B->insts.empty()) B->insts[0]->chunks = hc[0];  // batch total of chunks, reported once
    return ZETA_OK;
}

zeta_status engine_run(DeviceEngine *e, std::vector<Instance *> &batch, zeta_policy policy, zeta_path path,
                       std::string &err, double *ms_device) {
    cudaEvent_t ev0, ev1;
    CUDA_TRY(cudaSetDevice(e->device));
    CUDA_TRY(cudaEventCreate(&ev0));
    CUDA_TRY(cudaEventCreate(&ev1));
    CUDA_TRY(cudaEventRecord(ev0, e->stream));
    DeviceBatch *B = nullptr;
    zeta_status st = engine_prepare(e, batch, policy, path, &B, err);
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
    (void)path;
    CUDA_TRY(cudaSetDevice(e->device));
    if (s == 0 || c == 0 || s > kMaxS || c > kMaxC) { err = "s or c out of range"; return ZETA_ERR_ARG; }
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
    int grid = (int)std::min<uint32_t>(count, (uint32_t)e->sms * 4);
    uint64_t *d_scratch;
    if ((st = ensure(e, "hscratch", sizeof(uint64_t) * 2 * s * s * (size_t)grid, (void **)&d_scratch, err))) return st;
    size_t smem = (size_t)4 * s * c * sizeof(uint32_t);
    const int CPT = c <= 6 ? 2 : (c <= 12 ? 3 : 4);
    const void *kfn = CPT == 2 ? (const void *)k_horner_problems<2> : CPT == 3 ? (const void *)k_horner_problems<3> : (const void *)k_horner_problems<4>;
    CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (CPT == 2) k_horner_problems<2><<<grid, kThreads, smem, e->stream>>>(count, (int)s, (int)c, k, A, B, W, d_mods, d_scratch);
    else if (CPT == 3) k_horner_problems<3><<<grid, kThreads, smem, e->stream>>>(count, (int)s, (int)c, k, A, B, W, d_mods, d_scratch);
    else k_horner_problems<4><<<grid, kThreads, smem, e->stream>>>(count, (int)s, (int)c, k, A, B, W, d_mods, d_scratch);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(e->stream));
    return ZETA_OK;
}

}  // namespace zeta
