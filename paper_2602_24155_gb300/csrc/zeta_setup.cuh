// Device part of the host setup (included by zeta_kernels.cu after the modular
// arithmetic): right inverses over Z/q, q = p^M, for a batch of matrices --
// the section of the map of J_S (Prop. 3.3) and the final reduction's levels
// (Sec. 3.3 step (2)).
//
// Each job is an R x C matrix A of full row rank mod p, given by its nonzero
// entries (Montgomery form).  One CTA per job forms [A | I] (R x (C + R)) in
// global memory and runs Gauss-Jordan with unit pivots: for c = 0, 1, ... the
// first row at or below the current rank whose entry in column c is a unit
// (nonzero mod p) becomes the pivot row, is scaled to 1 and cleared from every
// other row.  Exact arithmetic and the same pivot rule as the host's
// elimination give the same matrix word for word.  Row k of the identity
// block is then the right inverse's row at the k-th pivot column; the kernel
// writes those R x R words and the pivot columns, the host places them.
namespace zeta {

struct SolveDesc {
    ModQ Q;
    uint64_t p;
    uint64_t aug;    // [A | I] in the work pool (row-major, R x W words)
    uint64_t out;    // R x R words in the output pool
    uint64_t nz;     // first of A's nonzeros in the entry pools
    uint32_t nnz;
    uint32_t R, C, W;
    uint32_t piv;    // first of the R pivot columns in the pivot pool
};

// a^{-1} mod q for a unit a in [1, q), q < 2^60 (extended Euclid; |t| stays below q).
__device__ inline uint64_t inv_mod_q(uint64_t a, uint64_t q) {
    int64_t r0 = (int64_t)q, r1 = (int64_t)a, t0 = 0, t1 = 1;
    while (r1) {
        const int64_t k = r0 / r1;
        int64_t tmp = r0 - k * r1;
        r0 = r1;
        r1 = tmp;
        tmp = t0 - k * t1;
        t0 = t1;
        t1 = tmp;
    }
    return t0 < 0 ? (uint64_t)(t0 + (int64_t)q) : (uint64_t)t0;
}

__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, const ModQ &Q) {
    return redc(a * b, mul_hi64(a, b), Q);
}

constexpr int kSolveThreads = 256;

// Grid-stride over the jobs.  Dynamic shared memory: the scaled pivot row (W words).
// nz_idx[e] = row * C + column of nonzero e; nz_val[e] its value (Montgomery form).
// rank_out[t] < R means A is not onto mod p (the job's output is then incomplete).
__global__ void __launch_bounds__(kSolveThreads) k_right_inverse(const SolveDesc *__restrict__ descs, uint32_t count,
                                                                 const uint32_t *__restrict__ nz_idx,
                                                                 const uint64_t *__restrict__ nz_val,
                                                                 uint64_t *__restrict__ work, uint64_t *__restrict__ out,
                                                                 int32_t *__restrict__ pivots, int32_t *__restrict__ rank_out) {
    extern __shared__ __align__(16) uint64_t s_prow[];
    __shared__ int s_piv;
    __shared__ uint64_t s_inv;
    const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kSolveThreads / 32;
    for (uint32_t t = blockIdx.x; t < count; t += gridDim.x) {
        const SolveDesc D = descs[t];
        const int R = (int)D.R, C = (int)D.C, W = (int)D.W;
        uint64_t *aug = work + D.aug;
        const uint64_t one = to_mont(1, D.Q);
        for (size_t e = tid; e < (size_t)R * W; e += kSolveThreads) aug[e] = 0;
        __syncthreads();
        for (uint32_t e = tid; e < D.nnz; e += kSolveThreads) {
            const uint32_t rc = nz_idx[D.nz + e];
            aug[(size_t)(rc / (uint32_t)C) * W + rc % (uint32_t)C] = nz_val[D.nz + e];
        }
        for (int r = tid; r < R; r += kSolveThreads) aug[(size_t)r * W + C + r] = one;
        __syncthreads();
        int rank = 0;
        for (int c = 0; c < C && rank < R; c++) {
            if (tid == 0) s_piv = R;
            __syncthreads();
            for (int i = rank + tid; i < R; i += kSolveThreads)
                if (redc(aug[(size_t)i * W + c], 0, D.Q) % D.p) atomicMin(&s_piv, i);
            __syncthreads();
            const int pr = s_piv;
            __syncthreads();  // every thread has read s_piv before the next column resets it
            if (pr == R) continue;  // no unit in this column: not a pivot column
            uint64_t *rk = aug + (size_t)rank * W;
            if (pr != rank) {
                uint64_t *rp = aug + (size_t)pr * W;
                for (int j = tid; j < W; j += kSolveThreads) {
                    const uint64_t x = rk[j];
                    rk[j] = rp[j];
                    rp[j] = x;
                }
            }
            __syncthreads();
            if (tid == 0) s_inv = to_mont(inv_mod_q(redc(rk[c], 0, D.Q), D.Q.q), D.Q);
            __syncthreads();
            const uint64_t inv = s_inv;
            for (int j = tid; j < W; j += kSolveThreads) {
                const uint64_t v = mont_mul(rk[j], inv, D.Q);
                rk[j] = v;
                s_prow[j] = v;
            }
            __syncthreads();
            // one warp per row: f = row[c] is read by every lane before any lane writes the row
            for (int i = warp; i < R; i += nwarps) {
                if (i == rank) continue;
                uint64_t *row = aug + (size_t)i * W;
                const uint64_t f = row[c];
                __syncwarp();
                if (!f) continue;
                for (int j = lane; j < W; j += 32) {
                    const uint64_t pj = s_prow[j];
                    if (pj) row[j] = submod(row[j], mont_mul(f, pj, D.Q), D.Q.q);
                }
            }
            if (tid == 0) pivots[D.piv + rank] = c;
            rank++;
            __syncthreads();
        }
        if (tid == 0) rank_out[t] = rank;
        for (size_t e = tid; e < (size_t)rank * R; e += kSolveThreads)
            out[D.out + e] = aug[(e / R) * W + C + e % R];
        __syncthreads();
    }
}

// Large matrices (a cubic fourfold's section: 6188 x 24206 words) on the whole GPU, one job at a time, two
// launches per column c: k_ri_pivot (one block) advances the rank past the previous column's pivot, finds the
// pivot row of column c, swaps it into place and scales it; k_ri_elim (every block, a warp per row) clears
// column c from the other rows with the pivot row staged in shared memory.  The same elimination as
// k_right_inverse, spread over blocks; the kernel boundaries order the columns.
struct SolveState {
    int32_t rank, found;
};

__global__ void __launch_bounds__(1024) k_ri_init(SolveDesc D, const uint32_t *__restrict__ nz_idx,
                                                  const uint64_t *__restrict__ nz_val, uint64_t *__restrict__ work,
                                                  SolveState *__restrict__ state) {
    uint64_t *aug = work + D.aug;
    const size_t stride = (size_t)gridDim.x * blockDim.x, t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (size_t e = t0; e < (size_t)D.R * D.W; e += stride) {
        const size_t r = e / D.W, c = e % D.W;
        aug[e] = c == D.C + r ? to_mont(1, D.Q) : 0;
    }
    if (t0 == 0) {
        state->rank = 0;
        state->found = 0;
    }
}

__global__ void __launch_bounds__(1024) k_ri_scatter(SolveDesc D, const uint32_t *__restrict__ nz_idx,
                                                     const uint64_t *__restrict__ nz_val, uint64_t *__restrict__ work) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D.nnz) return;
    const uint32_t rc = nz_idx[D.nz + e];
    work[D.aug + (size_t)(rc / D.C) * D.W + rc % D.C] = nz_val[D.nz + e];
}

__global__ void __launch_bounds__(1024) k_ri_pivot(SolveDesc D, int c, uint64_t *__restrict__ work,
                                                   int32_t *__restrict__ pivots, SolveState *__restrict__ state) {
    __shared__ int s_piv;
    __shared__ uint64_t s_inv;
    const int tid = (int)threadIdx.x, nt = (int)blockDim.x;
    const int R = (int)D.R, W = (int)D.W;
    const SolveState st = *state;
    const int rank = st.rank + st.found;  // the previous column's pivot row is in place
    __syncthreads();  // every thread has read the state before thread 0 rewrites it
    if (rank >= R) {
        if (tid == 0) *state = SolveState{rank, 0};
        return;
    }
    uint64_t *aug = work + D.aug;
    if (tid == 0) s_piv = R;
    __syncthreads();
    for (int i = rank + tid; i < R; i += nt)
        if (redc(aug[(size_t)i * W + c], 0, D.Q) % D.p) atomicMin(&s_piv, i);
    __syncthreads();
    const int pr = s_piv;
    if (pr == R) {
        if (tid == 0) *state = SolveState{rank, 0};
        return;
    }
    uint64_t *rk = aug + (size_t)rank * W;
    if (pr != rank) {
        uint64_t *rp = aug + (size_t)pr * W;
        for (int j = tid; j < W; j += nt) {
            const uint64_t x = rk[j];
            rk[j] = rp[j];
            rp[j] = x;
        }
    }
    __syncthreads();
    if (tid == 0) s_inv = to_mont(inv_mod_q(redc(rk[c], 0, D.Q), D.Q.q), D.Q);
    __syncthreads();
    const uint64_t inv = s_inv;
    for (int j = tid; j < W; j += nt) rk[j] = mont_mul(rk[j], inv, D.Q);
    if (tid == 0) {
        pivots[D.piv + rank] = c;
        *state = SolveState{rank, 1};
    }
}

// Dynamic shared memory: the pivot row (W words).  Block b clears rows [b RB, (b + 1) RB); a block none of whose
// rows has a nonzero entry in column c neither stages the pivot row nor touches memory again (most blocks, while
// the matrix is still sparse).
__global__ void __launch_bounds__(kSolveThreads) k_ri_elim(SolveDesc D, int c, uint64_t *__restrict__ work,
                                                           const SolveState *__restrict__ state) {
    extern __shared__ __align__(16) uint64_t s_prow[];
    const SolveState st = *state;
    if (!st.found) return;
    const int R = (int)D.R, W = (int)D.W, rank = st.rank;
    const int RB = (R + (int)gridDim.x - 1) / (int)gridDim.x;
    const int r0 = (int)blockIdx.x * RB, r1 = min(R, r0 + RB);
    uint64_t *aug = work + D.aug;
    int any = 0;
    for (int i = r0 + (int)threadIdx.x; i < r1; i += kSolveThreads)
        if (i != rank && aug[(size_t)i * W + c]) any = 1;
    if (!__syncthreads_or(any)) return;
    const uint64_t *rk = aug + (size_t)rank * W;
    for (int j = threadIdx.x; j < W; j += kSolveThreads) s_prow[j] = rk[j];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i = r0 + (int)(threadIdx.x >> 5); i < r1; i += kSolveThreads / 32) {
        if (i == rank) continue;
        uint64_t *row = aug + (size_t)i * W;
        const uint64_t f = row[c];
        __syncwarp();
        if (!f) continue;
        for (int j = lane; j < W; j += 32) {
            const uint64_t pj = s_prow[j];
            if (pj) row[j] = submod(row[j], mont_mul(f, pj, D.Q), D.Q.q);
        }
    }
}

__global__ void k_ri_out(SolveDesc D, const uint64_t *__restrict__ work, uint64_t *__restrict__ out,
                         const SolveState *__restrict__ state, int32_t *__restrict__ rank_out) {
    const SolveState st = *state;
    const int rank = st.rank + st.found;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    if (t0 == 0) *rank_out = rank;
    for (size_t e = t0; e < (size_t)rank * D.R; e += stride)
        out[D.out + e] = work[D.aug + (e / D.R) * D.W + D.C + e % D.R];
}

}  // namespace zeta
