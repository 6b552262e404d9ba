// Training and inference kernels of the direction-scoring network used by the
// learned reduction policy (zeta_learn.cpp).  A candidate direction is a row of
// kPolicyFeatures floats; the network is
//   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), score = h2 . w3 + b3
// (FP32, hidden width H <= 128).  A decision is a group of consecutive rows;
// the loss is the mean over groups of -log softmax(score)[label].
// Everything here is hand-written: one thread per row for the forward pass and
// the pre-activation gradients (weights staged in shared memory), one thread
// per parameter for the gradient sums over rows (deterministic, no atomics),
// one thread per group for the softmax, one per parameter for Adam (Kingma &
// Ba 2015).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "zeta_internal.h"

namespace zeta {

constexpr int kMlpMaxHidden = 128;

struct MlpView {
    int H;
    size_t oW1, ob1, oW2, ob2, ow3, ob3, count;
};

static MlpView mlp_view(int H) {
    const size_t F = kPolicyFeatures;
    MlpView v;
    v.H = H;
    v.oW1 = 0;
    v.ob1 = F * H;
    v.oW2 = v.ob1 + H;
    v.ob2 = v.oW2 + (size_t)H * H;
    v.ow3 = v.ob2 + H;
    v.ob3 = v.ow3 + H;
    v.count = v.ob3 + 1;
    return v;
}

// Forward: scores[r] and (optionally) the hidden activations for backward.
__global__ void k_mlp_forward(const float *__restrict__ params, int H, const float *__restrict__ X, size_t n,
                              float *__restrict__ scores, float *__restrict__ h1out, float *__restrict__ h2out) {
    extern __shared__ float sp[];
    const int F = kPolicyFeatures;
    const size_t cnt = (size_t)F * H + H + (size_t)H * H + H + H + 1;
    for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
    const float *W1 = sp, *b1 = W1 + F * H, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H, *b3 = w3 + H;
    for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (size_t)gridDim.x * blockDim.x) {
        float x[kPolicyFeatures];
        for (int i = 0; i < F; i++) x[i] = X[r * F + i];
        float h1[kMlpMaxHidden];
        for (int j = 0; j < H; j++) {
            float a = b1[j];
            for (int i = 0; i < F; i++) a = fmaf(x[i], W1[i * H + j], a);
            h1[j] = a > 0.f ? a : 0.f;
            if (h1out) h1out[r * H + j] = h1[j];
        }
        float out = b3[0];
        for (int j = 0; j < H; j++) {
            float a = b2[j];
            for (int i = 0; i < H; i++) a = fmaf(h1[i], W2[i * H + j], a);
            a = a > 0.f ? a : 0.f;
            if (h2out) h2out[r * H + j] = a;
            out = fmaf(a, w3[j], out);
        }
        scores[r] = out;
    }
}

// Softmax cross-entropy per group: dscore = (softmax - onehot(label)) / ngroups_total.
__global__ void k_mlp_softmax(const float *__restrict__ scores, const uint32_t *__restrict__ goff,
                              const uint32_t *__restrict__ labels, size_t g0, size_t g1, float inv_groups,
                              float *__restrict__ dscore, float *__restrict__ loss) {
    for (size_t g = g0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += (size_t)gridDim.x * blockDim.x) {
        const uint32_t a = goff[g], b = goff[g + 1];
        float mx = -INFINITY;
        for (uint32_t r = a; r < b; r++) mx = fmaxf(mx, scores[r]);
        float sum = 0.f;
        for (uint32_t r = a; r < b; r++) sum += expf(scores[r] - mx);
        const uint32_t lab = a + labels[g];
        for (uint32_t r = a; r < b; r++) dscore[r] = (expf(scores[r] - mx) / sum - (r == lab ? 1.f : 0.f)) * inv_groups;
        atomicAdd(loss, (logf(sum) + mx - scores[lab]) * inv_groups);
    }
}

// Backward, part 1 (one thread per row): the pre-activation gradients
//   d2[r, j] = [h2 > 0] ds[r] w3[j],  d1[r, i] = [h1 > 0] sum_j W2[i, j] d2[r, j].
__global__ void k_mlp_back_rows(const float *__restrict__ params, int H, const float *__restrict__ h1,
                                const float *__restrict__ h2, const float *__restrict__ dscore, size_t r0, size_t r1,
                                float *__restrict__ d1, float *__restrict__ d2) {
    extern __shared__ float sp[];
    const int F = kPolicyFeatures;
    const size_t cnt = (size_t)F * H + H + (size_t)H * H + H + H + 1;
    for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
    const float *W2 = sp + F * H + H, *w3 = W2 + H * H + H;
    for (size_t r = r0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < r1; r += (size_t)gridDim.x * blockDim.x) {
        const float ds = dscore[r];
        float g2[kMlpMaxHidden];
        for (int j = 0; j < H; j++) {
            g2[j] = h2[r * H + j] > 0.f ? ds * w3[j] : 0.f;
            d2[r * H + j] = g2[j];
        }
        for (int i = 0; i < H; i++) {
            float a = 0.f;
            for (int j = 0; j < H; j++) a = fmaf(W2[i * H + j], g2[j], a);
            d1[r * H + i] = h1[r * H + i] > 0.f ? a : 0.f;
        }
    }
}

// Backward, part 2: parameter gradients as a two-level sum, deterministic (no
// atomics).  Block row y takes the rows [r0 + y rchunk, r0 + (y+1) rchunk) of
// [r0, r1) (one thread per parameter) and writes its partial sums to
// part[y cnt + p]; k_mlp_sum_parts adds the partials in chunk order.
__global__ void k_mlp_back_params(int H, const float *__restrict__ X, const float *__restrict__ h1,
                                  const float *__restrict__ h2, const float *__restrict__ d1,
                                  const float *__restrict__ d2, const float *__restrict__ dscore, size_t r0_all,
                                  size_t r1_all, size_t rchunk, float *__restrict__ part) {
    const int F = kPolicyFeatures;
    const size_t ob1 = (size_t)F * H, oW2 = ob1 + H, ob2 = oW2 + (size_t)H * H, ow3 = ob2 + H, ob3 = ow3 + H;
    const size_t cnt = ob3 + 1;
    const size_t r0 = r0_all + (size_t)blockIdx.y * rchunk;
    const size_t r1 = min(r1_all, r0 + rchunk);
    float *out = part + (size_t)blockIdx.y * cnt;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < cnt; p += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        if (p < ob1) {
            const int f = (int)(p / H), i = (int)(p % H);
            for (size_t r = r0; r < r1; r++) acc = fmaf(X[r * F + f], d1[r * H + i], acc);
        } else if (p < oW2) {
            const int i = (int)(p - ob1);
            for (size_t r = r0; r < r1; r++) acc += d1[r * H + i];
        } else if (p < ob2) {
            const int i = (int)((p - oW2) / H), j = (int)((p - oW2) % H);
            for (size_t r = r0; r < r1; r++) acc = fmaf(h1[r * H + i], d2[r * H + j], acc);
        } else if (p < ow3) {
            const int j = (int)(p - ob2);
            for (size_t r = r0; r < r1; r++) acc += d2[r * H + j];
        } else if (p < ob3) {
            const int j = (int)(p - ow3);
            for (size_t r = r0; r < r1; r++) acc = fmaf(dscore[r], h2[r * H + j], acc);
        } else {
            for (size_t r = r0; r < r1; r++) acc += dscore[r];
        }
        out[p] = acc;
    }
}

__global__ void k_mlp_sum_parts(const float *__restrict__ part, size_t nchunks, size_t cnt, float *__restrict__ grad) {
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < cnt; p += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (size_t c = 0; c < nchunks; c++) acc += part[c * cnt + p];
        grad[p] += acc;
    }
}

// Row chunks of the parameter gradient: at most kMlpMaxChunks, at least 32 rows each.
constexpr size_t kMlpMaxChunks = 256;
inline size_t mlp_rchunk(size_t rows) { return std::max<size_t>(32, (rows + kMlpMaxChunks - 1) / kMlpMaxChunks); }

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       size_t n, float lr, float b1, float b2, float b1t, float b2t, float eps) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        m[i] = b1 * m[i] + (1.f - b1) * gi;
        v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
        const float mh = m[i] / (1.f - b1t), vh = v[i] / (1.f - b2t);
        p[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}

namespace {

struct DevMem {
    std::vector<void *> ptrs;
    ~DevMem() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T **out, size_t count) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, sizeof(T) * std::max<size_t>(count, 1));
        if (e == cudaSuccess) ptrs.push_back(p);
        *out = (T *)p;
        return e;
    }
};

#define MLP_TRY(expr)                                              \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) {                                   \
            cudaGetLastError();                                    \
            return ZETA_ERR_DEVICE;                                \
        }                                                          \
    } while (0)

zeta_status check_hidden(uint32_t hidden) {
    return (hidden >= 1 && hidden <= (uint32_t)kMlpMaxHidden) ? ZETA_OK : ZETA_ERR_ARG;
}

size_t fwd_smem(int H) { return sizeof(float) * mlp_view(H).count; }

// The weights staged in shared memory exceed the 48 KB default above width 110 (75.8 KB at 128): raise the
// limit of the two kernels that stage them to what the widest network needs.
cudaError_t mlp_kernel_attributes() {
    const int bytes = (int)fwd_smem(kMlpMaxHidden);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)k_mlp_back_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

}  // namespace

// Forward + softmax + backward of one range of groups; grad (device) accumulated.
static zeta_status mlp_step(int H, const float *d_params, const float *d_X, const uint32_t *d_goff,
                            const uint32_t *d_lab, const std::vector<uint32_t> &goff, size_t g0, size_t g1,
                            float inv_groups, float *d_scores, float *d_h1, float *d_h2, float *d_ds, float *d_d1,
                            float *d_d2, float *d_grad, float *d_loss, float *d_part, cudaStream_t st) {
    const size_t r0 = goff[g0], r1 = goff[g1];
    const size_t rows = r1 - r0;
    if (rows == 0) return ZETA_OK;
    const int T = 128;
    const int blocks = (int)std::min<size_t>((rows + T - 1) / T, 4096);
    k_mlp_forward<<<blocks, T, fwd_smem(H), st>>>(d_params, H, d_X + r0 * kPolicyFeatures, rows, d_scores + r0,
                                                   d_h1 + r0 * H, d_h2 + r0 * H);
    MLP_TRY(cudaGetLastError());
    const int gb = (int)std::min<size_t>((g1 - g0 + T - 1) / T, 4096);
    k_mlp_softmax<<<gb, T, 0, st>>>(d_scores, d_goff, d_lab, g0, g1, inv_groups, d_ds, d_loss);
    MLP_TRY(cudaGetLastError());
    k_mlp_back_rows<<<blocks, T, fwd_smem(H), st>>>(d_params, H, d_h1, d_h2, d_ds, r0, r1, d_d1, d_d2);
    MLP_TRY(cudaGetLastError());
    const size_t cnt = mlp_view(H).count;
    const size_t rchunk = mlp_rchunk(rows), nchunks = (rows + rchunk - 1) / rchunk;
    k_mlp_back_params<<<dim3((unsigned)((cnt + T - 1) / T), (unsigned)nchunks), T, 0, st>>>(
        H, d_X, d_h1, d_h2, d_d1, d_d2, d_ds, r0, r1, rchunk, d_part);
    MLP_TRY(cudaGetLastError());
    k_mlp_sum_parts<<<(int)((cnt + T - 1) / T), T, 0, st>>>(d_part, nchunks, cnt, d_grad);
    MLP_TRY(cudaGetLastError());
    return ZETA_OK;
}

}  // namespace zeta

using namespace zeta;

extern "C" size_t zeta_mlp_param_count(uint32_t hidden) { return policy_param_count((int)hidden); }

extern "C" zeta_status zeta_mlp_init(uint32_t hidden, uint64_t seed, float *params) {
    if (!params || check_hidden(hidden)) return ZETA_ERR_ARG;
    const MlpView v = mlp_view((int)hidden);
    uint64_t s = seed;
    auto next = [&]() {  // splitmix64 (Steele, Lea, Flood 2014)
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uni = [&](float a) { return (float)((next() >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * a; };
    const float a1 = std::sqrt(6.f / (kPolicyFeatures + hidden)), a2 = std::sqrt(6.f / (2.f * hidden)),
                a3 = std::sqrt(6.f / (hidden + 1.f));
    std::memset(params, 0, sizeof(float) * v.count);
    for (size_t i = 0; i < (size_t)kPolicyFeatures * hidden; i++) params[v.oW1 + i] = uni(a1);
    for (size_t i = 0; i < (size_t)hidden * hidden; i++) params[v.oW2 + i] = uni(a2);
    for (size_t i = 0; i < hidden; i++) params[v.ow3 + i] = uni(a3);
    return ZETA_OK;
}

extern "C" zeta_status zeta_mlp_forward(zeta_ctx *ctx, uint32_t hidden, const float *params, const float *X, size_t n,
                                        float *scores) {
    (void)ctx;
    if (!params || (n && (!X || !scores)) || check_hidden(hidden)) return ZETA_ERR_ARG;
    if (n == 0) return ZETA_OK;
    const int H = (int)hidden;
    DevMem mem;
    float *dp, *dX, *ds;
    MLP_TRY(mlp_kernel_attributes());
    MLP_TRY(mem.alloc(&dp, mlp_view(H).count));
    MLP_TRY(mem.alloc(&dX, n * kPolicyFeatures));
    MLP_TRY(mem.alloc(&ds, n));
    MLP_TRY(cudaMemcpy(dp, params, sizeof(float) * mlp_view(H).count, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(dX, X, sizeof(float) * n * kPolicyFeatures, cudaMemcpyHostToDevice));
    const int T = 128, blocks = (int)std::min<size_t>((n + T - 1) / T, 4096);
    k_mlp_forward<<<blocks, T, fwd_smem(H)>>>(dp, H, dX, n, ds, nullptr, nullptr);
    MLP_TRY(cudaGetLastError());
    MLP_TRY(cudaMemcpy(scores, ds, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return ZETA_OK;
}

extern "C" zeta_status zeta_mlp_grad(zeta_ctx *ctx, uint32_t hidden, const float *params, const float *X,
                                     const uint32_t *group_off, const uint32_t *labels, size_t ngroups, float *grad,
                                     float *loss) {
    (void)ctx;
    if (!params || !grad || !group_off || (ngroups && (!X || !labels)) || check_hidden(hidden)) return ZETA_ERR_ARG;
    const int H = (int)hidden;
    const MlpView v = mlp_view(H);
    std::vector<uint32_t> goff(group_off, group_off + ngroups + 1);
    const size_t n = goff[ngroups];
    for (size_t g = 0; g < ngroups; g++)
        if (goff[g + 1] <= goff[g] || labels[g] >= goff[g + 1] - goff[g]) return ZETA_ERR_ARG;
    DevMem mem;
    float *dp, *dX, *dsc, *dh1, *dh2, *dds, *dg, *dl, *dd1, *dd2;
    uint32_t *dgo, *dlab;
    MLP_TRY(mlp_kernel_attributes());
    MLP_TRY(mem.alloc(&dd1, n * H));
    MLP_TRY(mem.alloc(&dd2, n * H));
    MLP_TRY(mem.alloc(&dp, v.count));
    MLP_TRY(mem.alloc(&dX, n * kPolicyFeatures));
    MLP_TRY(mem.alloc(&dsc, n));
    MLP_TRY(mem.alloc(&dh1, n * H));
    MLP_TRY(mem.alloc(&dh2, n * H));
    MLP_TRY(mem.alloc(&dds, n));
    MLP_TRY(mem.alloc(&dg, v.count));
    MLP_TRY(mem.alloc(&dl, 1));
    MLP_TRY(mem.alloc(&dgo, ngroups + 1));
    MLP_TRY(mem.alloc(&dlab, ngroups));
    float *dpart;
    MLP_TRY(mem.alloc(&dpart, kMlpMaxChunks * v.count));
    MLP_TRY(cudaMemcpy(dp, params, sizeof(float) * v.count, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(dX, X, sizeof(float) * n * kPolicyFeatures, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(dgo, goff.data(), sizeof(uint32_t) * goff.size(), cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(dlab, labels, sizeof(uint32_t) * ngroups, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemset(dg, 0, sizeof(float) * v.count));
    MLP_TRY(cudaMemset(dl, 0, sizeof(float)));
    MLP_TRY(cudaMemset(dds, 0, sizeof(float) * n));
    zeta_status st = mlp_step(H, dp, dX, dgo, dlab, goff, 0, ngroups, 1.f / (float)std::max<size_t>(ngroups, 1), dsc,
                              dh1, dh2, dds, dd1, dd2, dg, dl, dpart, 0);
    if (st) return st;
    MLP_TRY(cudaMemcpy(grad, dg, sizeof(float) * v.count, cudaMemcpyDeviceToHost));
    if (loss) MLP_TRY(cudaMemcpy(loss, dl, sizeof(float), cudaMemcpyDeviceToHost));
    return ZETA_OK;
}

extern "C" zeta_status zeta_mlp_train(zeta_ctx *ctx, uint32_t hidden, float *params, const float *X,
                                      const uint32_t *group_off, const uint32_t *labels, size_t ngroups,
                                      uint32_t epochs, uint32_t batch_groups, float lr, float *final_loss) {
    (void)ctx;
    if (!params || !group_off || (ngroups && (!X || !labels)) || !batch_groups || check_hidden(hidden))
        return ZETA_ERR_ARG;
    const int H = (int)hidden;
    const MlpView v = mlp_view(H);
    std::vector<uint32_t> goff(group_off, group_off + ngroups + 1);
    const size_t n = goff[ngroups];
    for (size_t g = 0; g < ngroups; g++)
        if (goff[g + 1] <= goff[g] || labels[g] >= goff[g + 1] - goff[g]) return ZETA_ERR_ARG;
    DevMem mem;
    float *dp, *dX, *dsc, *dh1, *dh2, *dds, *dg, *dm, *dv, *dl, *dd1, *dd2;
    uint32_t *dgo, *dlab;
    MLP_TRY(mlp_kernel_attributes());
    MLP_TRY(mem.alloc(&dd1, n * H));
    MLP_TRY(mem.alloc(&dd2, n * H));
    MLP_TRY(mem.alloc(&dp, v.count));
    MLP_TRY(mem.alloc(&dX, n * kPolicyFeatures));
    MLP_TRY(mem.alloc(&dsc, n));
    MLP_TRY(mem.alloc(&dh1, n * H));
    MLP_TRY(mem.alloc(&dh2, n * H));
    MLP_TRY(mem.alloc(&dds, n));
    MLP_TRY(mem.alloc(&dg, v.count));
    MLP_TRY(mem.alloc(&dm, v.count));
    MLP_TRY(mem.alloc(&dv, v.count));
    MLP_TRY(mem.alloc(&dl, 1));
    MLP_TRY(mem.alloc(&dgo, ngroups + 1));
    MLP_TRY(mem.alloc(&dlab, ngroups));
    float *dpart;
    MLP_TRY(mem.alloc(&dpart, kMlpMaxChunks * v.count));
    MLP_TRY(cudaMemcpy(dp, params, sizeof(float) * v.count, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(dX, X, sizeof(float) * n * kPolicyFeatures, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(dgo, goff.data(), sizeof(uint32_t) * goff.size(), cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(dlab, labels, sizeof(uint32_t) * ngroups, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemset(dm, 0, sizeof(float) * v.count));
    MLP_TRY(cudaMemset(dv, 0, sizeof(float) * v.count));
    const float b1 = 0.9f, b2 = 0.999f;
    float b1t = 1.f, b2t = 1.f, last = 0.f;
    for (uint32_t ep = 0; ep < epochs; ep++) {
        MLP_TRY(cudaMemset(dl, 0, sizeof(float)));
        for (size_t g0 = 0; g0 < ngroups; g0 += batch_groups) {
            const size_t g1 = std::min(ngroups, g0 + batch_groups);
            MLP_TRY(cudaMemset(dg, 0, sizeof(float) * v.count));
            zeta_status st = mlp_step(H, dp, dX, dgo, dlab, goff, g0, g1, 1.f / (float)(g1 - g0), dsc, dh1, dh2, dds,
                                      dd1, dd2, dg, dl, dpart, 0);
            if (st) return st;
            b1t *= b1;
            b2t *= b2;
            k_adam<<<(int)std::min<size_t>((v.count + 255) / 256, 1024), 256>>>(dp, dg, dm, dv, v.count, lr, b1, b2,
                                                                                   b1t, b2t, 1e-8f);
            MLP_TRY(cudaGetLastError());
        }
        MLP_TRY(cudaMemcpy(&last, dl, sizeof(float), cudaMemcpyDeviceToHost));
        last /= (float)((ngroups + batch_groups - 1) / batch_groups);  // mean of the batch means
    }
    MLP_TRY(cudaMemcpy(params, dp, sizeof(float) * v.count, cudaMemcpyDeviceToHost));
    if (final_loss) *final_loss = last;
    return ZETA_OK;
}
