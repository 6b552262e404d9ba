// Cluster executor of the reduction plan for large step matrices (included by
// zeta_kernels.cu after the plan structures).
//
// An instance whose s x s step matrix does not fit one SM's shared memory
// (quartic K3 surfaces: s = 220, cubic threefolds: s = 495) is reduced by one
// thread-block cluster of CL CTAs.  CTA t of the cluster owns rows
// [t R, t R + R) of the step matrices (R = ceil(s / CL)): it builds its rows
// of A and M(k-1) = R_{U-v,v} from the section (Prop. 3.3), keeps its rows of
// M in shared memory (A in global memory, read once per step) and, for every
// step of Algorithm 2 (Sec. 3.2), computes its rows of M W and writes them
// into the W buffer of every CTA of the cluster through distributed shared
// memory (st.shared::cluster).  One cluster barrier (release/acquire) per step
// separates the steps; M <- M - A runs between the arrive and the wait.
// Moves 2 (merges into the next phase) and the pole-order-n numerators are
// written row slice by row slice, so no two CTAs write the same word.
//
// Arithmetic (a row r and four columns per work item):
//  - q < 2^56: M entries m (Montgomery form) and W entries w as two 28-bit
//    limbs; four 32x32->64 multiply-adds per product, partial sums below
//    256 * 2^56 = 2^64 over blocks of at most 256 terms, each block folded to
//    a 128-bit X < 256 q^2 < q 2^64 and reduced once (REDC, R = 2^64).
//  - 2^56 <= q < 2^60: the 20-bit x 30-bit split of horner_block (six
//    multiply-adds per product).
// When a step has few work items, the j range of each item is split between
// P = 2, 4 or 8 lanes of a warp whose residues are added with shuffles.
namespace zeta {

constexpr int kClusterMinS = 128;     // instances with larger s run on clusters
constexpr int kClThreads = 384;

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_sync() {
    cl_arrive();
    cl_wait();
}
__device__ __forceinline__ uint32_t cl_map(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_st_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint32_t cl_ld_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Limb packing of W entries: 28-bit limbs for q < 2^56, else 30-bit limbs.
__device__ __forceinline__ uint2 cl_pack(uint64_t v, int lb) {
    return make_uint2((uint32_t)v & ((1u << lb) - 1u), (uint32_t)(v >> lb));
}
__device__ __forceinline__ uint64_t cl_unpack(uint2 w, int lb) { return ((uint64_t)w.y << lb) | w.x; }

// Residues of four output columns of one work item over j in [jb, je).
template <bool L28>
__device__ __forceinline__ void cl_item_sums(const uint64_t *__restrict__ Ms, int nrows, int rl, const uint2 *in,
                                             int cs, int c0, int jb, int je, const ModQ &Q, uint64_t (&v)[4]) {
    v[0] = v[1] = v[2] = v[3] = 0;
    if (L28) {
        const uint32_t M28 = (1u << 28) - 1u;
        for (int j0 = jb; j0 < je; j0 += 256) {
            const int j1 = min(je, j0 + 256);
            uint64_t S[4][4];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int t = 0; t < 4; t++) S[a][t] = 0;
            const uint64_t *mp = Ms + (size_t)j0 * nrows + rl;
            const uint4 *wp = reinterpret_cast<const uint4 *>(in + (size_t)j0 * cs + c0);
            const int wstride = cs / 2;
#pragma unroll 2
            for (int j = j0; j < j1; j++) {
                const uint64_t m = *mp;
                mp += nrows;
                const uint32_t m0 = (uint32_t)m & M28, m1 = (uint32_t)(m >> 28);
                const uint4 wa = wp[0], wb = wp[1];
                wp += wstride;
                madw(S[0][0], m0, wa.x); madw(S[0][1], m0, wa.y); madw(S[0][2], m1, wa.x); madw(S[0][3], m1, wa.y);
                madw(S[1][0], m0, wa.z); madw(S[1][1], m0, wa.w); madw(S[1][2], m1, wa.z); madw(S[1][3], m1, wa.w);
                madw(S[2][0], m0, wb.x); madw(S[2][1], m0, wb.y); madw(S[2][2], m1, wb.x); madw(S[2][3], m1, wb.y);
                madw(S[3][0], m0, wb.z); madw(S[3][1], m0, wb.w); madw(S[3][2], m1, wb.z); madw(S[3][3], m1, wb.w);
            }
#pragma unroll
            for (int a = 0; a < 4; a++) {
                // X = S00 + (S01 + S10) 2^28 + S11 2^56 < 256 q^2 < q 2^64
                uint64_t lo = S[a][0], hi = 0;
                add128(lo, hi, S[a][1] << 28); hi += S[a][1] >> 36;
                add128(lo, hi, S[a][2] << 28); hi += S[a][2] >> 36;
                add128(lo, hi, S[a][3] << 56); hi += S[a][3] >> 8;
                v[a] = addmod(v[a], redc(lo, hi, Q), Q.q);
            }
        }
    } else {
        const uint32_t M20 = (1u << 20) - 1u;
        uint64_t S[4][6];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int t = 0; t < 6; t++) S[a][t] = 0;
        const uint64_t *mp = Ms + (size_t)jb * nrows + rl;
        const uint4 *wp = reinterpret_cast<const uint4 *>(in + (size_t)jb * cs + c0);
        const int wstride = cs / 2;
#pragma unroll 2
        for (int j = jb; j < je; j++) {
            const uint64_t m = *mp;
            mp += nrows;
            const uint32_t m0 = (uint32_t)m & M20, m1 = (uint32_t)(m >> 20) & M20, m2 = (uint32_t)(m >> 40);
            const uint4 wa = wp[0], wb = wp[1];
            wp += wstride;
            madw(S[0][0], m0, wa.x); madw(S[0][1], m0, wa.y); madw(S[0][2], m1, wa.x);
            madw(S[0][3], m1, wa.y); madw(S[0][4], m2, wa.x); madw(S[0][5], m2, wa.y);
            madw(S[1][0], m0, wa.z); madw(S[1][1], m0, wa.w); madw(S[1][2], m1, wa.z);
            madw(S[1][3], m1, wa.w); madw(S[1][4], m2, wa.z); madw(S[1][5], m2, wa.w);
            madw(S[2][0], m0, wb.x); madw(S[2][1], m0, wb.y); madw(S[2][2], m1, wb.x);
            madw(S[2][3], m1, wb.y); madw(S[2][4], m2, wb.x); madw(S[2][5], m2, wb.y);
            madw(S[3][0], m0, wb.z); madw(S[3][1], m0, wb.w); madw(S[3][2], m1, wb.z);
            madw(S[3][3], m1, wb.w); madw(S[3][4], m2, wb.z); madw(S[3][5], m2, wb.w);
        }
#pragma unroll
        for (int a = 0; a < 4; a++) v[a] = fold_partials(S[a], Q);
    }
}

// k steps of Algorithm 2 by the cluster: this CTA's rows [row0, row0 + nrows)
// of M(k-1) (Montgomery form, [j][rl] with row stride nrows) in Ms, the same
// rows of A in Ag (global); W (s x cs limb pairs, every row) in W0 or W1
// (cur); returns the buffer holding the result.  Every CTA of the cluster
// calls it with the same s, c, k.
template <bool L28>
__device__ int cl_horner(int s, int c, int k, int row0, int nrows, uint64_t *Ms, const uint64_t *__restrict__ Ag,
                         uint2 *W0, uint2 *W1, int cur, const ModQ &Q, uint32_t ncta) {
    const int cs = pad4(c);
    const int items = nrows > 0 ? nrows * (cs / 4) : 0;
    const int nt = (int)blockDim.x;
    int P = 1;
    while (P < 8 && items * P * 2 <= nt) P *= 2;
    const int ipw = 32 / P;  // items per warp when the j range is split
    const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
    const int part = P > 1 ? lane / ipw : 0;
    const int lb = L28 ? 28 : 30;
    const int nms = nrows > 0 ? nrows * s : 0;
    for (int step = 0; step < k; step++) {
        const uint2 *in = cur ? W1 : W0;
        const uint32_t out_s = smem_u32(cur ? W0 : W1);
        for (int base = 0; base < items; base += (P > 1 ? items : nt)) {
            const int it = P > 1 ? warp * ipw + lane % ipw : base + (int)threadIdx.x;
            const bool valid = it < items;
            if (P == 1 && !valid) break;
            const int rl = valid ? it % nrows : 0;
            const int c0 = valid ? (it / nrows) * 4 : 0;
            const int jb = valid ? part * s / P : 0, je = valid ? (part + 1) * s / P : 0;
            uint64_t v[4];
            cl_item_sums<L28>(Ms, nrows, rl, in, cs, c0, jb, je, Q, v);
            if (P > 1) {
#pragma unroll
                for (int a = 0; a < 4; a++)
                    for (int off = 16; off >= ipw; off >>= 1)
                        v[a] = addmod(v[a], __shfl_xor_sync(0xffffffffu, v[a], off), Q.q);
            }
            if (valid && part == 0) {
                const uint2 r0 = cl_pack(v[0], lb), r1 = cl_pack(v[1], lb), r2 = cl_pack(v[2], lb),
                            r3 = cl_pack(v[3], lb);
                const uint4 lo4 = make_uint4(r0.x, r0.y, r1.x, r1.y), hi4 = make_uint4(r2.x, r2.y, r3.x, r3.y);
                const uint32_t a = out_s + (uint32_t)(((row0 + rl) * cs + c0) * 8);
                for (uint32_t t = 0; t < ncta; t++) {
                    const uint32_t ra = cl_map(a, t);
                    cl_st_v4(ra, lo4);
                    cl_st_v4(ra + 16, hi4);
                }
            }
        }
        __syncthreads();  // this CTA's reads of M for the step are done
        cl_arrive();
        if (step + 1 < k) {
            // M <- M - A: A streamed from global memory 16 bytes at a time, four loads in flight per thread
            const int n2 = nms >> 1;
            const uint4 *A4 = reinterpret_cast<const uint4 *>(Ag);
            uint4 *M4 = reinterpret_cast<uint4 *>(Ms);
            for (int base = (int)threadIdx.x; base < n2; base += 4 * nt) {
                uint4 av[4];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (base + u * nt < n2) av[u] = __ldcg(&A4[base + u * nt]);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int e = base + u * nt;
                    if (e >= n2) break;
                    uint4 m = M4[e];
                    const uint64_t lo = submod(((uint64_t)m.y << 32) | m.x, ((uint64_t)av[u].y << 32) | av[u].x, Q.q);
                    const uint64_t hi = submod(((uint64_t)m.w << 32) | m.z, ((uint64_t)av[u].w << 32) | av[u].z, Q.q);
                    M4[e] = make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
                }
            }
            if ((nms & 1) && threadIdx.x == 0) Ms[nms - 1] = submod(Ms[nms - 1], Ag[nms - 1], Q.q);
        }
        __syncthreads();
        cl_wait();        // every CTA's rows of the new W have landed here
        cur ^= 1;
    }
    return cur;
}

// Shared memory of the cluster executor: M rows (R x s), two W buffers
// (s x cs, 16-byte aligned), column map (32) and column indices (s).
__host__ __device__ inline size_t cl_w_offset(int s, int R) { return ((size_t)R * s * sizeof(uint64_t) + 127) & ~(size_t)127; }
__host__ __device__ inline size_t cl_smem(int s, int c, int R) {
    return cl_w_offset(s, R) + (size_t)2 * s * pad4(c) * sizeof(uint2) + (size_t)(32 + s) * sizeof(int) + 64;
}

// Persistent plan executor on clusters.  Clusters take instances from the
// queue (largest work first); CTA rank 0 draws and the others read its draw
// through distributed shared memory.  secT: the sections transposed (column
// gamma holds rows (i, nu) contiguously), in Montgomery form.
__global__ void __launch_bounds__(kClThreads, 1) k_execute_cluster(
    const DInst *__restrict__ insts, const DTab *__restrict__ tabs, const int32_t *__restrict__ tabpool,
    const uint64_t *__restrict__ secT, const DChain *__restrict__ chains, const Term *__restrict__ terms,
    const uint32_t *__restrict__ phase_pool, const DEntry *__restrict__ entries, const DChunk *__restrict__ chunks,
    const uint32_t *__restrict__ order, uint32_t ninst, uint32_t *__restrict__ queue,
    uint64_t *__restrict__ ascratch, size_t a_stride, uint64_t *__restrict__ blocks, size_t blocks_stride,
    uint64_t *__restrict__ Hout, size_t h_stride, unsigned long long *__restrict__ counters,
    unsigned long long *__restrict__ stamps) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int sU[kMaxVars], sv[kMaxVars], s_nlive;
    __shared__ uint32_t s_item;
    const uint32_t rank = cl_rank(), ncta = cl_size();
    uint64_t *Ag = ascratch + (size_t)blockIdx.x * a_stride;
    uint64_t *bufA = blocks + (size_t)cl_id() * blocks_stride;
    uint64_t *bufB = bufA + blocks_stride / 2;
    unsigned long long my_chunks = 0, my_steps = 0;
    const uint32_t item_addr0 = cl_map(smem_u32(&s_item), 0);
    // device latency (as in k_execute): launch start, and each instance's start and end
    if (threadIdx.x == 0) atomicMin(&stamps[2 * (size_t)ninst], global_ns());
    while (true) {
        if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        cl_sync();
        const uint32_t itx = cl_ld_u32(item_addr0);
        const uint32_t inst = itx < ninst ? order[itx] : 0;
        const DInst I = insts[inst];
        const int s = (int)I.s, b = (int)I.b, nv = (int)I.nv, n = (int)I.n, d = (int)I.d;
        uint64_t *Hg = Hout + (size_t)inst * h_stride;
        if (itx < ninst) {
            const int hb = (int)I.h_rows * b;
            const int per = (hb + (int)ncta - 1) / (int)ncta;
            for (int e = (int)rank * per + (int)threadIdx.x; e < min(hb, ((int)rank + 1) * per); e += blockDim.x)
                Hg[e] = 0;
        }
        cl_sync();  // every CTA has read the draw (rank 0 may draw again only after the instance)
        if (itx >= ninst) break;
        if (rank == 0 && threadIdx.x == 0) stamps[2 * inst] = global_ns();
        const DTab T = tabs[I.tab];
        const int32_t *monoS = tabpool + T.monoS_off;
        const int32_t *secrow = tabpool + T.secrow_off;
        const uint64_t *SecT = secT + I.sec_off;
        const uint32_t *ph = phase_pool + I.phase_off;
        const int R = (s + (int)ncta - 1) / (int)ncta;
        const int row0 = (int)rank * R;
        const int nrows = max(0, min(R, s - row0));
        // shared memory of this instance (cl_smem(s, b, R) bytes): M rows, W0, W1, column map, column indices
        uint64_t *Ms = reinterpret_cast<uint64_t *>(smem_raw);
        uint2 *W0 = reinterpret_cast<uint2 *>(smem_raw + cl_w_offset(s, R));
        uint2 *W1 = W0 + (size_t)s * pad4(b);
        int *colmap = reinterpret_cast<int *>(W1 + (size_t)s * pad4(b));
        int *colidx = colmap + 32;
        const bool l28 = I.Q.q < (1ull << 56);
        const int lb = l28 ? 28 : 30;
        int res_buf = 1;  // buffer holding the last result; the first entry forms its W in the other
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
                // This CTA's rows of W in the buffer the previous entry's last step read from (every CTA
                // passed that step's barrier, so no CTA reads it any more): the arrival block's live columns
                // or 0, plus the start terms on these rows ((row, column) is unique within a chain), then
                // sent to every other CTA of the cluster.
                const int src = res_buf ^ 1;
                uint2 *Wf = src ? W1 : W0;
                for (int e = threadIdx.x; e < nrows * cs; e += blockDim.x) {
                    const int j = row0 + e / cs, lc = e % cs;
                    uint64_t val = 0;
                    if (E.arrival >= 0 && lc < c) val = cur[(size_t)E.arrival * s * b + (size_t)j * b + colmap[lc]];
                    Wf[j * cs + lc] = cl_pack(val, lb);
                }
                __syncthreads();
                if (E.start_chain >= 0) {
                    const DChain C = chains[I.chain_base + E.start_chain];
                    for (uint32_t t = C.term_begin + threadIdx.x; t < C.term_end; t += blockDim.x) {
                        const Term tm = terms[t];
                        if ((int)tm.row < row0 || (int)tm.row >= row0 + nrows) continue;
                        int lc = 0;
                        while (colmap[lc] != (int)tm.col) lc++;
                        const int e = (int)tm.row * cs + lc;
                        Wf[e] = cl_pack(addmod(cl_unpack(Wf[e], lb), tm.coeff, I.Q.q), lb);
                    }
                }
                __syncthreads();
                {
                    const uint32_t base = smem_u32(Wf) + (uint32_t)(row0 * cs * 8);
                    const uint4 *own = reinterpret_cast<const uint4 *>(Wf + row0 * cs);
                    for (int e = threadIdx.x; e < nrows * cs / 2; e += blockDim.x) {
                        const uint4 val = own[e];
                        for (uint32_t t = 0; t < ncta; t++)
                            if (t != rank) cl_st_v4(cl_map(base + 16u * (uint32_t)e, t), val);
                    }
                }
                cl_arrive();  // W's rows are sent; the first chunk's matrices are built while the others finish
                int cur_buf = src;
                for (uint32_t ci = E.chunk_begin; ci < E.chunk_end; ci++) {
                    const DChunk CH = chunks[I.chunk_base + ci];
                    const int k = CH.k;
                    if (threadIdx.x < (unsigned)nv) sv[threadIdx.x] = CH.v[threadIdx.x];
                    __syncthreads();
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
                    // this CTA's rows of A R and M(k-1) R = R_{U-v,v} R, [j][rl]
                    for (int e = threadIdx.x; e < nrows * s; e += blockDim.x) {
                        const int j = e / nrows, rl = e - j * nrows, r = row0 + rl;
                        const int col = colidx[j];
                        uint64_t aL = 0, mL = 0, mH = 0;
                        if (col >= 0) {
                            const uint64_t *sc = SecT + (size_t)col * I.sec_rows;
                            for (int i = 0; i < nv; i++) {
                                const int row = secrow[i * s + r];
                                if (row < 0) continue;
                                const uint64_t val = __ldg(&sc[row]);
                                aL += val * (uint64_t)sv[i];  // < d q < 2^63
                                const uint64_t wm = (uint64_t)(sU[i] - sv[i] + monoS[r * nv + i]);
                                add128(mL, mH, val * wm);
                                mH += mul_hi64(val, wm);
                            }
                        }
                        while (aL >= I.Q.q) aL -= I.Q.q;
                        Ag[e] = aL;
                        Ms[e] = reduce128(mL, mH, I.Q);
                    }
                    __syncthreads();
                    if (ci == E.chunk_begin) cl_wait();  // every CTA's rows of W have landed here
                    cur_buf = l28 ? cl_horner<true>(s, c, k, row0, nrows, Ms, Ag, W0, W1, cur_buf, I.Q, ncta)
                                  : cl_horner<false>(s, c, k, row0, nrows, Ms, Ag, W0, W1, cur_buf, I.Q, ncta);
                    if (threadIdx.x == 0) {
                        for (int t = 0; t < nv; t++) sU[t] -= k * sv[t];
                        if (rank == 0) {
                            my_chunks++;
                            my_steps += k;
                        }
                    }
                    __syncthreads();
                }
                if (E.chunk_begin == E.chunk_end) cl_wait();
                res_buf = cur_buf;
                const uint2 *Rw = cur_buf ? W1 : W0;
                if (E.dest < 0) {
                    // pole order n: this CTA's rows of x^U g / x^S added into H (distinct rows, distinct h)
                    const int hdeg = d * n - n - 1;
                    for (int e = threadIdx.x; e < nrows * c; e += blockDim.x) {
                        const int j = row0 + e / c, lc = e % c;
                        const uint64_t val = cl_unpack(Rw[j * cs + lc], lb);
                        if (!val) continue;
                        int g[kMaxVars];
                        bool ok = true;
                        for (int t = 0; t < nv; t++) {
                            g[t] = sU[t] + monoS[j * nv + t] - 1;
                            if (g[t] < 0) ok = false;
                        }
                        if (!ok) continue;
                        const int h = dev_rank(g, nv, hdeg);
                        const int col = colmap[lc];
                        Hg[h * b + col] = addmod(Hg[h * b + col], val, I.Q.q);
                    }
                } else {
                    // move 2: this CTA's rows stored (first contribution) or added into the next phase's block
                    uint64_t *dst = nxt + (size_t)E.dest * s * b;
                    if (E.flags & 1u) {
                        for (int e = threadIdx.x; e < nrows * b; e += blockDim.x) dst[(size_t)row0 * b + e] = 0;
                        __syncthreads();
                    }
                    for (int e = threadIdx.x; e < nrows * c; e += blockDim.x) {
                        const int j = row0 + e / c, lc = e % c;
                        const uint64_t val = cl_unpack(Rw[j * cs + lc], lb);
                        uint64_t &slot = dst[(size_t)j * b + colmap[lc]];
                        slot = addmod(slot, val, I.Q.q);
                    }
                }
                // the result is read (the next entry starts by overwriting the entry's state)
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) atomicMax(&stamps[2 * inst + 1], global_ns());  // the cluster's last CTA to finish
    }
    if (rank == 0 && threadIdx.x == 0) {
        atomicAdd(&counters[0], my_chunks);
        atomicAdd(&counters[1], my_steps);
    }
}

}  // namespace zeta
