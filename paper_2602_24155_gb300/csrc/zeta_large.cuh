// Whole-GPU plan executor for large step matrices (included by zeta_kernels.cu
// after the plan structures): one instance at a time, the host walking its
// plan (phases, entries, chunks) and every kernel spread over all SMs.  Built
// for the cubic fourfolds (s = C(15, 5) = 3003, whose M(y) and A take 72 MB
// each) and for bases of more than 32 columns (quintic surfaces: b = 52), it
// runs any instance with q < 2^56, s <= 4096 and b <= 64.
//
// Layouts (global memory): M, A row-major [r s + j] (Montgomery form, R = 2^64;
// 32-bit words when q < 2^32, so that M and A of a cubic fourfold, 36 MB each,
// stay in L2 across the steps of a chunk);
// W, V column-major [col s + j] (ordinary residues); the phase blocks and H as
// the persistent executors' ([j b + col] and [h b + col]).
//
// Per chunk (Sec. 3.4 move 1, Algorithm 2): k_lg_gen forms A and M(k-1) =
// R_{U-v,v} from the section (Prop. 3.3); then k reduction steps, each one
// k_lg_step launch (V = M W; M <- M - A), the kernel boundary being the only
// synchronisation between steps.
namespace zeta {

constexpr int kLgWarps = 8;  // rows (one per warp) per block of k_lg_step
constexpr int kLgMaxCpt = 8; // columns per k_lg_step pass

struct LgVec {
    int32_t x[kMaxVars];
};

struct LgCols {
    int32_t col[64];  // basis column of live column lc
    int32_t lc[64];   // live column of basis column col, or -1
    int32_t c;
};

// Column of Sec read for column j of the chunk's matrices: rank_kappa(v + e_j - 1), or -1.
__global__ void k_lg_colidx(int s, int nv, int kappa, const int32_t *__restrict__ monoS, LgVec v,
                            int32_t *__restrict__ colidx) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= s) return;
    int g[kMaxVars];
    bool ok = true;
    for (int t = 0; t < nv; t++) {
        g[t] = v.x[t] + monoS[j * nv + t] - 1;
        if (g[t] < 0) ok = false;
    }
    colidx[j] = ok ? dev_rank(g, nv, kappa) : -1;
}

// A R and M(k-1) R = R_{U-v,v} R (row r, column j):
//   A[r,j] = sum_i v_i Sec[(i, omega_r - 1_S + e_i), v + e_j - 1],
//   M[r,j] = sum_i (U_i - v_i + e_{r,i}) Sec[(i, omega_r - 1_S + e_i), v + e_j - 1],
// Sec held as Sec R mod q (row-major, sec_cols words per row).  One thread per
// entry, j fastest: consecutive threads read one Sec row at increasing columns.
// T: the storage word of Sec, M and A (uint32_t when q < 2^32, else uint64_t).
template <typename T>
__global__ void __launch_bounds__(256) k_lg_gen(int s, int nv, uint32_t sec_cols, const int32_t *__restrict__ monoS,
                                                const int32_t *__restrict__ secrow, const int32_t *__restrict__ colidx,
                                                const T *__restrict__ Sec, LgVec U, LgVec v, ModQ Q,
                                                T *__restrict__ M, T *__restrict__ A) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)s * s) return;
    const int r = (int)(e / (size_t)s), j = (int)(e % (size_t)s);
    const int col = colidx[j];
    uint64_t aL = 0, mL = 0, mH = 0;
    if (col >= 0) {
        uint64_t val[kMaxVars];  // all section reads in flight before the first is used
#pragma unroll
        for (int i = 0; i < kMaxVars; i++) {
            val[i] = 0;
            if (i < nv) {
                const int row = secrow[i * s + r];
                if (row >= 0) val[i] = (uint64_t)__ldg(&Sec[(size_t)row * sec_cols + col]);
            }
        }
#pragma unroll
        for (int i = 0; i < kMaxVars; i++)
            if (i < nv) {
                aL += val[i] * (uint64_t)v.x[i];  // < d q < 2^63
                const uint64_t wm = (uint64_t)(U.x[i] - v.x[i] + monoS[r * nv + i]);
                add128(mL, mH, val[i] * wm);
                mH += mul_hi64(val[i], wm);
            }
    }
    while (aL >= Q.q) aL -= Q.q;
    A[e] = (T)aL;
    M[e] = (T)reduce128(mL, mH, Q);
}

// One reduction step for columns [0, c) of W and V (c <= CPT; the caller offsets
// the pointers for later column groups) and, when `last`, M <- M - A.  One warp
// per row r, lanes over j.  q < 2^56: M's and W's entries split into 28-bit limbs,
// four mad.wide.u32 per product into 64-bit partial sums (a lane adds at most
// ceil(s/32) <= 128 products below 2^56); the 128-bit total X < 128 q^2 < q 2^64 is
// reduced once per lane (REDC gives M W mod q, M being in Montgomery form) and
// the lanes' residues are added over the warp.
template <int CPT, typename T>
__global__ void __launch_bounds__(kLgWarps * 32) k_lg_step(int s, int c, const uint64_t *__restrict__ W,
                                                           uint64_t *__restrict__ V, T *__restrict__ M,
                                                           const T *__restrict__ A, ModQ Q, int last) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * kLgWarps + (threadIdx.x >> 5);
    if (r >= s) return;  // the whole warp leaves together
    constexpr uint32_t MASK = (1u << 28) - 1u;
    uint64_t S[CPT][4];
#pragma unroll
    for (int t = 0; t < CPT; t++) S[t][0] = S[t][1] = S[t][2] = S[t][3] = 0;
    T *Mr = M + (size_t)r * s;
    const T *Ar = A + (size_t)r * s;
#pragma unroll 4
    for (int j = lane; j < s; j += 32) {
        const uint64_t m = (uint64_t)Mr[j];
        if (last) Mr[j] = (T)submod(m, (uint64_t)__ldg(&Ar[j]), Q.q);
        const uint32_t m0 = (uint32_t)m & MASK, m1 = (uint32_t)(m >> 28);
#pragma unroll
        for (int t = 0; t < CPT; t++) {
            if (t < c) {
                const uint64_t w = __ldg(&W[(size_t)t * s + j]);
                const uint32_t w0 = (uint32_t)w & MASK, w1 = (uint32_t)(w >> 28);
                madw(S[t][0], m0, w0);
                madw(S[t][1], m0, w1);
                madw(S[t][2], m1, w0);
                madw(S[t][3], m1, w1);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < CPT; t++) {
        if (t >= c) break;
        uint64_t lo = S[t][0], hi = 0;
        add128(lo, hi, S[t][1] << 28);
        hi += S[t][1] >> 36;
        add128(lo, hi, S[t][2] << 28);
        hi += S[t][2] >> 36;
        add128(lo, hi, S[t][3] << 56);
        hi += S[t][3] >> 8;
        uint64_t x = redc(lo, hi, Q);
#pragma unroll
        for (int off = 16; off; off >>= 1) x = addmod(x, __shfl_xor_sync(0xffffffffu, x, off), Q.q);
        if (lane == 0) V[(size_t)t * s + r] = x;
    }
}

// Narrow moduli (q < 2^26: the cubic fourfolds at relative precision 1, q = 7^9): products of two residues are
// below 2^52, so a 64-bit sum of up to 4096 of them needs no limbs -- one mad.wide.u32 per product.  M and A
// are 32-bit words in rows of stride sp (s rounded up to 4, the padding zero), read 16 bytes at a time.

// A R and M(k-1) R as above, from Sec R^2 mod q (32-bit words): each is one REDC of a sum below 2^48.  Grid:
// (sp / 256 rounded up, s); block y is row r, threads run over j; every product is one mad.wide.u32 (a section word
// below 2^26 times a weight below 2^16) and every index fits 32 bits (the section has under 2^32 words).
__global__ void __launch_bounds__(256) k_lg_gen_narrow(int s, int sp, int nv, uint32_t sec_cols,
                                                       const int32_t *__restrict__ monoS,
                                                       const int32_t *__restrict__ secrow,
                                                       const int32_t *__restrict__ colidx,
                                                       const uint32_t *__restrict__ SecRR, LgVec U, LgVec v, ModQ Q,
                                                       uint32_t *__restrict__ M, uint32_t *__restrict__ A) {
    const int r = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= sp) return;
    uint64_t aL = 0, mL = 0;
    const int col = j < s ? colidx[j] : -1;
    if (col >= 0) {
        // every section read issued before the first is used (the reads are independent; issued one after the
        // other the kernel waits nv memory latencies per entry)
        uint32_t val[kMaxVars];
#pragma unroll
        for (int i = 0; i < kMaxVars; i++) {
            val[i] = 0;
            if (i < nv) {
                const int row = __ldg(&secrow[i * s + r]);
                if (row >= 0) val[i] = __ldg(&SecRR[(uint32_t)row * sec_cols + (uint32_t)col]);
            }
        }
#pragma unroll
        for (int i = 0; i < kMaxVars; i++)
            if (i < nv) {
                madw(aL, val[i], (uint32_t)v.x[i]);
                madw(mL, val[i], (uint32_t)(U.x[i] - v.x[i] + __ldg(&monoS[r * nv + i])));
            }
    }
    const size_t e = (size_t)r * sp + j;
    A[e] = (uint32_t)redc(aL, 0, Q);
    M[e] = (uint32_t)redc(mL, 0, Q);
}

// Step t of a chunk for columns [0, c) (c <= CPT).  kLgSplit warps per row, each lane four consecutive j per
// 16-byte load, the warps' residues added through shared memory; W staged in shared memory as 32-bit words,
// kLgTileJ columns j at a time.  W, V: 64-bit words, column stride sp.  Two forms:
//  WRITE = false: V = M(k-1) W - t (A W), tR = t R mod q; M is only read (two products per entry: chunks with one
//                 or two columns, where the step is bound by reading M and A);
//  WRITE = true:  V = M W with the current M(k-1-t), and, when `last`, M <- M - A (one product per entry: chunks
//                 with three or more columns, where the products dominate).
constexpr int kLgTileJ = 1024;
constexpr int kLgSplit = 2;  // warps per row of the narrow step (a row of 3003 words per warp leaves 20 warps per SM)

template <int CPT, bool WRITE>
__global__ void __launch_bounds__(kLgWarps * 32) k_lg_step_narrow(int s, int sp, int c, const uint64_t *__restrict__ W,
                                                                  uint64_t *__restrict__ V, uint32_t *__restrict__ M,
                                                                  const uint32_t *__restrict__ A, ModQ Q, uint64_t tR,
                                                                  int last) {
    __shared__ __align__(16) uint32_t sW[CPT][kLgTileJ];
    __shared__ uint64_t s_part[kLgWarps][CPT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * (kLgWarps / kLgSplit) + warp / kLgSplit, part = warp % kLgSplit;
    const bool row_ok = r < s;  // a warp past the last row still helps stage W
    uint64_t SM[CPT], SA[CPT];
#pragma unroll
    for (int t = 0; t < CPT; t++) SM[t] = SA[t] = 0;
    uint4 *Mr = reinterpret_cast<uint4 *>(M + (size_t)(row_ok ? r : 0) * sp);
    const uint4 *Ar = reinterpret_cast<const uint4 *>(A + (size_t)(row_ok ? r : 0) * sp);
    for (int j0 = 0; j0 < sp; j0 += kLgTileJ) {
        const int jn = min(kLgTileJ, sp - j0);  // a multiple of 4
        __syncthreads();  // the previous tile is consumed
        for (int e = threadIdx.x; e < c * jn; e += kLgWarps * 32) {
            const int t = e / jn, j = e - t * jn;
            sW[t][j] = (uint32_t)W[(size_t)t * sp + j0 + j];
        }
        __syncthreads();
        if (row_ok) {
            // four 16-byte loads of M and A in flight per lane: the step is bound by memory latency otherwise
#pragma unroll 4
            for (int q4 = lane + 32 * part; q4 < (jn >> 2); q4 += 32 * kLgSplit) {
                const int g = (j0 >> 2) + q4;
                const uint4 m = Mr[g];
                uint4 a = make_uint4(0, 0, 0, 0);
                if (!WRITE || last) a = __ldg(&Ar[g]);
#pragma unroll
                for (int t = 0; t < CPT; t++) {
                    if (t < c) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(&sW[t][4 * q4]);
                        madw(SM[t], m.x, w.x);
                        madw(SM[t], m.y, w.y);
                        madw(SM[t], m.z, w.z);
                        madw(SM[t], m.w, w.w);
                        if (!WRITE) {
                            madw(SA[t], a.x, w.x);
                            madw(SA[t], a.y, w.y);
                            madw(SA[t], a.z, w.z);
                            madw(SA[t], a.w, w.w);
                        }
                    }
                }
                if (WRITE && last)
                    Mr[g] = make_uint4((uint32_t)submod(m.x, a.x, Q.q), (uint32_t)submod(m.y, a.y, Q.q),
                                       (uint32_t)submod(m.z, a.z, Q.q), (uint32_t)submod(m.w, a.w, Q.q));
            }
        }
    }
#pragma unroll
    for (int t = 0; t < CPT; t++) {
        if (t >= c) break;
        uint64_t z = redc(SM[t], 0, Q);  // M W mod q
        if (!WRITE) {
            const uint64_t y = redc(SA[t], 0, Q);  // A W mod q
            z = submod(z, redc(y * tR, mul_hi64(y, tR), Q), Q.q);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) z = addmod(z, __shfl_xor_sync(0xffffffffu, z, off), Q.q);
        if (lane == 0) s_part[warp][t] = z;
    }
    __syncthreads();  // the row's other warps have written their part
    if (!row_ok || part != 0 || lane >= c) return;
    uint64_t z = s_part[warp][lane];
#pragma unroll
    for (int k = 1; k < kLgSplit; k++) z = addmod(z, s_part[warp + k][lane], Q.q);
    V[(size_t)lane * sp + r] = z;
}

// W = the live columns of the arrival block (or 0 without one).
__global__ void k_lg_form(int s, int ws, int b, LgCols cm, const uint64_t *__restrict__ block, uint64_t *__restrict__ W) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)cm.c * s) return;
    const int lc = (int)(e / (size_t)s), j = (int)(e % (size_t)s);
    W[(size_t)lc * ws + j] = block ? block[(size_t)j * b + cm.col[lc]] : 0;
}

// The start terms of a chain (Prop. 2.1 after Tweak): (row, column) is unique within a chain.
__global__ void k_lg_terms(int ws, LgCols cm, const Term *__restrict__ terms, uint32_t begin, uint32_t end,
                           uint64_t *__restrict__ W, uint64_t q) {
    const uint32_t t = begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= end) return;
    const Term tm = terms[t];
    const int lc = tm.col < 64 ? cm.lc[tm.col] : -1;
    if (lc < 0) return;  // a term always lands on a live column of its entry
    uint64_t &w = W[(size_t)lc * ws + tm.row];
    w = addmod(w, tm.coeff, q);
}

// Move 2: store (first contribution; the other columns cleared) or add the result into the next phase's block.
__global__ void k_lg_merge(int s, int ws, int b, LgCols cm, const uint64_t *__restrict__ R, uint64_t *__restrict__ dst,
                           int first, uint64_t q) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)s * b) return;
    const int j = (int)(e / (size_t)b), col = (int)(e % (size_t)b);
    const int lc = cm.lc[col];
    if (lc < 0) {
        if (first) dst[e] = 0;
        return;
    }
    const uint64_t v = R[(size_t)lc * ws + j];
    dst[e] = first ? v : addmod(dst[e], v, q);
}

// Pole order n: H[rank(U + e_j - 1), col] += R[j, col] (x^U g / x^S on the numerator monomials; j -> U + e_j - 1
// is one to one, so no two threads meet).
__global__ void k_lg_numer(int s, int ws, int b, int nv, int hdeg, LgVec U, const int32_t *__restrict__ monoS,
                           LgCols cm, const uint64_t *__restrict__ R, uint64_t *__restrict__ H, uint64_t q) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)cm.c * s) return;
    const int lc = (int)(e / (size_t)s), j = (int)(e % (size_t)s);
    const uint64_t val = R[(size_t)lc * ws + j];
    if (!val) return;
    int g[kMaxVars];
    for (int t = 0; t < nv; t++) {
        g[t] = U.x[t] + monoS[j * nv + t] - 1;
        if (g[t] < 0) return;  // cannot carry a coefficient on a valid path
    }
    uint64_t &h = H[(size_t)dev_rank(g, nv, hdeg) * b + cm.col[lc]];
    h = addmod(h, val, q);
}

}  // namespace zeta
