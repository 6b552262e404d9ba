// C ABI of the library (declared in include/zeta.h).  Marshalling, host
// thread pool for the per-instance setup, and the device engine calls.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "zeta_internal.h"

using namespace zeta;

struct zeta_ctx {
    DeviceEngine *engine = nullptr;
    std::string error;
    unsigned threads = 1;
    std::map<std::pair<uint32_t, uint32_t>, zeta_tuning> tuned;  // zeta_autotune's choice per (n, d)
};

// ZETA_PATH_AUTO: the recorded choice for the instances' (n, d) (all equal),
// else the vector path with the default block.
static void resolve_path(const zeta_ctx *ctx, const std::vector<Instance *> &batch, zeta_options &o) {
    if (o.path != ZETA_PATH_AUTO) return;
    o.path = ZETA_PATH_VECTOR;
    o.block_threads = 0;
    if (batch.empty()) return;
    const uint32_t n = batch[0]->n, d = batch[0]->d;
    for (const Instance *X : batch)
        if (X->n != n || X->d != d) return;
    auto it = ctx->tuned.find({n, d});
    if (it == ctx->tuned.end()) return;
    const zeta_tuning &t = it->second;
    o.path = (zeta_path)t.cand_path[t.best];
    o.block_threads = t.cand_threads[t.best];
}

static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void parallel_for(size_t count, unsigned threads, const std::function<void(size_t)> &fn) {
    if (count == 0) return;
    threads = (unsigned)std::min<size_t>(std::max(1u, threads), count);
    if (threads == 1) {
        for (size_t i = 0; i < count; i++) fn(i);
        return;
    }
    std::atomic<size_t> next(0);
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < threads; t++)
        pool.emplace_back([&]() {
            for (size_t i = next++; i < count; i = next++) fn(i);
        });
    for (auto &th : pool) th.join();
}

static void fill_stats(const Instance &X, zeta_stats *st, double ms_device) {
    if (!st) return;
    std::memset(st, 0, sizeof(*st));
    st->status = (int32_t)X.status;
    st->b = X.b;
    st->r = X.r;
    st->M = X.M;
    for (int i = 0; i < 8; i++) st->N[i] = X.N[i];
    st->s = X.s;
    st->eps = X.eps;
    st->chains = X.chains.size();
    st->terms = X.nterms;
    st->chunks = X.chunks;
    st->steps = X.steps;
    st->column_steps = X.column_steps;
    st->ms_host_setup = X.ms_setup;
    st->ms_device = ms_device;
    st->ms_host_finish = X.ms_finish;
    st->ms_dev_start = X.ms_dev_start;
    st->ms_dev_end = X.ms_dev_end;
}

static uint64_t step_side(uint32_t n, uint32_t d);

static zeta_options default_options() {
    zeta_options o;
    std::memset(&o, 0, sizeof(o));
    o.policy = ZETA_POLICY_DEPTH_FIRST;
    o.path = ZETA_PATH_VECTOR;
    return o;
}

extern "C" {

zeta_status zeta_create(zeta_ctx **out, int device, void *cuda_stream) {
    if (!out) return ZETA_ERR_ARG;
    *out = nullptr;
    zeta_ctx *c = new (std::nothrow) zeta_ctx();
    if (!c) return ZETA_ERR_OOM;
    std::string err;
    c->engine = engine_create(device, cuda_stream, err);
    if (!c->engine) {
        delete c;
        return ZETA_ERR_DEVICE;
    }
    c->threads = std::max(1u, std::thread::hardware_concurrency());
    *out = c;
    return ZETA_OK;
}

zeta_status zeta_destroy(zeta_ctx *ctx) {
    if (!ctx) return ZETA_OK;
    engine_destroy(ctx->engine);
    delete ctx;
    return ZETA_OK;
}

const char *zeta_last_error(const zeta_ctx *ctx) {
    if (!ctx) return "null context";
    return ctx->error.c_str();
}

zeta_status zeta_query(const zeta_hypersurface *hs, const zeta_options *opt, uint32_t *b, uint32_t *r,
                       uint32_t *M, uint32_t *s) {
    if (!hs) return ZETA_ERR_ARG;
    zeta_options o = opt ? *opt : default_options();
    Instance X;
    zeta_status st = prepare_instance(hs, &o, false, X);
    if (st) return st;
    if (b) *b = X.b;
    if (r) *r = X.r;
    if (M) *M = X.M;
    if (s) *s = X.s;
    return ZETA_OK;
}

static zeta_status run_one(zeta_ctx *ctx, const zeta_hypersurface *hs, const zeta_options *opt, Instance &X,
                           double *ms_dev) {
    zeta_options o = opt ? *opt : default_options();
    // C(dn, n) > 512: the setup's right inverses on the device (the host refuses them)
    const bool big = hs && step_side(hs->n, hs->d) > 512;
    zeta_status st = prepare_instance(hs, &o, true, X, big);
    X.net.w = o.policy_weights;
    X.net.hidden = (int)o.policy_hidden;
    if (!st && X.solves_pending) {
        std::vector<SolveJob *> jobs;
        std::vector<uint64_t> qs, ps;
        for (SolveJob &J : X.solves)
            if (J.R) {
                jobs.push_back(&J);
                qs.push_back(X.q);
                ps.push_back(X.p);
            }
        st = engine_solve(ctx->engine, jobs, qs, ps, ctx->error, nullptr);
        if (st) return st;
        st = prepare_complete(X);
    }
    if (!st) st = schedule_policy(X, o.policy);
    if (st) { ctx->error = X.error; return st; }
    std::vector<Instance *> batch{&X};
    if (X.s > 512 || X.b > 32 || (o.flags & ZETA_FLAG_WHOLE_GPU)) {
        uint64_t launches = 0;
        st = engine_run_large(ctx->engine, batch, ctx->error, ms_dev, &launches, now_ms());
    } else {
        resolve_path(ctx, batch, o);
        st = engine_run(ctx->engine, batch, o.policy, o.path, o.block_threads, ctx->error, ms_dev);
    }
    if (st) return st;
    st = (o.flags & ZETA_FLAG_Y_ONLY) ? finish_y_only(X) : finish_instance(X);
    if (st) { ctx->error = X.error; return st; }
    return ZETA_OK;
}

zeta_status zeta_frobenius(zeta_ctx *ctx, const zeta_hypersurface *hs, const zeta_options *opt, uint64_t *F_out,
                           uint64_t *Y_out, zeta_stats *stats) {
    if (!ctx || !hs || !F_out) return ZETA_ERR_ARG;
    Instance X;
    double ms = 0;
    zeta_status st = run_one(ctx, hs, opt, X, &ms);
    if (st) return st;
    if (!X.F.empty()) std::memcpy(F_out, X.F.data(), sizeof(uint64_t) * X.F.size());
    else std::memset(F_out, 0, sizeof(uint64_t) * X.b * X.b);
    if (Y_out) std::memcpy(Y_out, X.Y.data(), sizeof(uint64_t) * X.Y.size());
    fill_stats(X, stats, ms);
    return ZETA_OK;
}

static void write_coeff(int64_t *dst, i128 v) {
    dst[0] = (int64_t)(uint64_t)((u128)v & 0xFFFFFFFFFFFFFFFFull);
    dst[1] = (int64_t)(v >> 64);
}

zeta_status zeta_charpoly(zeta_ctx *ctx, const zeta_hypersurface *hs, const zeta_options *opt, int64_t *P_out,
                          zeta_stats *stats) {
    if (!ctx || !hs || !P_out) return ZETA_ERR_ARG;
    Instance X;
    double ms = 0;
    zeta_status st = run_one(ctx, hs, opt, X, &ms);
    if (st) return st;
    for (uint32_t i = 0; i <= X.b; i++) write_coeff(P_out + 2 * i, i < X.P.size() ? X.P[i] : 0);
    fill_stats(X, stats, ms);
    return ZETA_OK;
}

}  // extern "C"

struct zeta_batch_plan {
    std::vector<Instance> inst;
    std::vector<Instance *> ok;
    std::vector<Instance *> large;  // one at a time on the whole-GPU executor (s > 512, b > 32, ZETA_FLAG_WHOLE_GPU)
    zeta_options opt;
    DeviceBatch *dev = nullptr;
    double ms_setup = 0, ms_device = 0, ms_large = 0;
    double t_run = 0;               // host steady clock (ms) at the last zeta_batch_run
    uint64_t large_launches = 0;
    bool launched = false, large_done = false;
};

// The instances of the whole-GPU executor, after the persistent launch was enqueued.
static zeta_status run_large(zeta_ctx *ctx, zeta_batch_plan *P) {
    if (P->large_done) return ZETA_OK;
    P->large_done = true;
    double ms = 0;
    uint64_t launches = 0;
    zeta_status st = engine_run_large(ctx->engine, P->large, ctx->error, &ms, &launches, P->t_run ? P->t_run : now_ms());
    if (st) return st;
    P->ms_large += ms;
    P->large_launches += launches;
    return ZETA_OK;
}

extern "C" {

}  // extern "C"

// zeta_batch_prepare on a given lane of the engine (0: the context's stream, 1: the engine's second stream).
static zeta_status batch_prepare_lane(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count, const zeta_options *opt,
                                      int lane, zeta_batch_plan **out, Instance *begun = nullptr);

// C(dn, n), the side of the step matrices (0 when out of range).
static uint64_t step_side(uint32_t n, uint32_t d) {
    if (n < 1 || n > 16 || d < 2 || d > 64) return 0;
    uint64_t r = 1;
    for (uint32_t i = 1; i <= n; i++) r = r * (uint64_t)(d * n - n + i) / i;
    return r;
}

// The setup's right inverses go to the device for batches holding an instance with s > 128 (there
// the host's Gauss-Jordan is most of the setup: about 2 s for a cubic threefold), unless a flag
// chooses; plane curves keep them on the host, whose setup is hidden behind the previous launch.
static bool wants_device_setup(const zeta_options &o, const zeta_hypersurface *hs, size_t count) {
    if (o.flags & ZETA_FLAG_HOST_SETUP) return false;
    if (o.flags & ZETA_FLAG_DEVICE_SETUP) return true;
    for (size_t i = 0; i < count; i++)
        if (step_side(hs[i].n, hs[i].d) > 128) return true;
    return false;
}

// Host setup of X[0..count) up to the right inverses (in parallel), then the right inverses of all
// of them in one device launch.  prepare_complete finishes each instance.
static zeta_status begin_on_device(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count, const zeta_options &o,
                                   Instance *X, double *ms_solve) {
    parallel_for(count, ctx->threads, [&](size_t i) {
        X[i].net.w = o.policy_weights;
        X[i].net.hidden = (int)o.policy_hidden;
        prepare_instance(&hs[i], &o, true, X[i], true);
    });
    std::vector<SolveJob *> jobs;
    std::vector<uint64_t> qs, ps;
    for (size_t i = 0; i < count; i++) {
        if (X[i].status != ZETA_OK || !X[i].solves_pending) continue;
        for (SolveJob &J : X[i].solves)
            if (J.R) {
                jobs.push_back(&J);
                qs.push_back(X[i].q);
                ps.push_back(X[i].p);
            }
    }
    return engine_solve(ctx->engine, jobs, qs, ps, ctx->error, ms_solve);
}

extern "C" {

zeta_status zeta_batch_prepare(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count, const zeta_options *opt,
                               zeta_batch_plan **out) {
    return batch_prepare_lane(ctx, hs, count, opt, 0, out);
}

}  // extern "C"

static zeta_status batch_prepare_lane(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count, const zeta_options *opt,
                                      int lane, zeta_batch_plan **out, Instance *begun) {
    if (!ctx || !out || (!hs && count)) return ZETA_ERR_ARG;
    *out = nullptr;
    zeta_batch_plan *P = new (std::nothrow) zeta_batch_plan();
    if (!P) return ZETA_ERR_OOM;
    P->opt = opt ? *opt : default_options();
    P->inst.resize(count);
    double t0 = now_ms();
    const bool device = !begun && wants_device_setup(P->opt, hs, count);
    if (begun) {
        for (size_t i = 0; i < count; i++) P->inst[i] = std::move(begun[i]);
    } else if (device) {
        zeta_status st = begin_on_device(ctx, hs, count, P->opt, P->inst.data(), nullptr);
        if (st) { delete P; return st; }
    }
    parallel_for(count, ctx->threads, [&](size_t i) {
        Instance &X = P->inst[i];
        if (!begun && !device) {
            X.net.w = P->opt.policy_weights;
            X.net.hidden = (int)P->opt.policy_hidden;
            if (prepare_instance(&hs[i], &P->opt, true, X) != ZETA_OK) return;
        } else if (X.status != ZETA_OK || (X.solves_pending && prepare_complete(X) != ZETA_OK)) {
            return;
        }
        schedule_policy(X, P->opt.policy);
    });
    for (auto &X : P->inst)
        if (X.status == ZETA_OK) P->ok.push_back(&X);
        else if (ctx->error.empty()) ctx->error = X.error;
    P->ms_setup = now_ms() - t0;
    std::vector<Instance *> small;
    for (Instance *X : P->ok)
        if (X->s > 512 || X->b > 32 || (P->opt.flags & ZETA_FLAG_WHOLE_GPU)) P->large.push_back(X);
        else small.push_back(X);
    if (!small.empty()) {
        resolve_path(ctx, small, P->opt);
        zeta_status st = engine_prepare(ctx->engine, small, P->opt.policy, P->opt.path, P->opt.block_threads, lane,
                                        &P->dev, ctx->error);
        if (st) { delete P; return st; }
    }
    *out = P;
    return ZETA_OK;
}

extern "C" {

zeta_status zeta_batch_run(zeta_ctx *ctx, zeta_batch_plan *P) {
    if (!ctx || !P) return ZETA_ERR_ARG;
    // every call runs the batch again (repeated launches of resident inputs are how a batch is timed)
    P->t_run = now_ms();
    if (P->dev) {
        P->launched = true;
        zeta_status st = engine_launch(ctx->engine, P->dev, ctx->error);
        if (st) return st;
    }
    P->large_done = false;
    return run_large(ctx, P);
}

zeta_status zeta_batch_finish(zeta_ctx *ctx, zeta_batch_plan *P, int64_t *P_out, size_t stride,
                              zeta_stats *per_instance, zeta_stats *total) {
    if (!ctx || !P || (!P_out && !P->inst.empty())) return ZETA_ERR_ARG;
    for (Instance *X : P->ok)
        if ((size_t)X->b + 1 > stride) return ZETA_ERR_ARG;
    if (P->dev && !P->launched) {
        P->launched = true;
        zeta_status st = engine_launch(ctx->engine, P->dev, ctx->error);
        if (st) return st;
    }
    {
        zeta_status st = run_large(ctx, P);
        if (st) return st;
    }
    if (P->dev) {
        zeta_status st = engine_collect(ctx->engine, P->dev, ctx->error);
        if (st) return st;
    }
    double t2 = now_ms();
    bool y_only = (P->opt.flags & ZETA_FLAG_Y_ONLY) != 0;
    parallel_for(P->ok.size(), ctx->threads, [&](size_t i) {
        if (y_only) finish_y_only(*P->ok[i]);
        else finish_instance(*P->ok[i]);
    });
    double t3 = now_ms();
    zeta_stats agg;
    std::memset(&agg, 0, sizeof(agg));
    for (size_t i = 0; i < P->inst.size(); i++) {
        Instance &X = P->inst[i];
        if (X.status == ZETA_OK) {
            for (uint32_t t = 0; t <= X.b; t++)
                write_coeff(P_out + 2 * (i * stride + t), t < X.P.size() ? X.P[t] : 0);
        } else if (ctx->error.empty()) {
            ctx->error = X.error;
        }
        if (per_instance) fill_stats(X, &per_instance[i], 0);
        if (X.status == ZETA_OK) {
            agg.chains += X.chains.size();
            agg.terms += X.nterms;
            agg.chunks += X.chunks;
            agg.steps += X.steps;
            agg.column_steps += X.column_steps;
        }
    }
    agg.ms_host_setup = P->ms_setup;
    agg.ms_host_finish = t3 - t2;
    engine_batch_timing(P->dev, &agg.ms_kernel, &agg.kernel_launches, &agg.bytes_h2d, &agg.bytes_d2h);
    agg.ms_kernel += P->ms_large;
    agg.kernel_launches += P->large_launches;
    if (total) *total = agg;
    return ZETA_OK;
}

zeta_status zeta_batch_release(zeta_batch_plan *P) {
    if (!P) return ZETA_OK;
    engine_release(P->dev);
    delete P;
    return ZETA_OK;
}

zeta_status zeta_batch(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count, const zeta_options *opt,
                       int64_t *P_out, size_t stride, zeta_stats *per_instance, zeta_stats *total) {
    if (!ctx || (!hs && count) || (!P_out && count)) return ZETA_ERR_ARG;
    // Pipelined: the host setup of sub-batch i+1 runs while the GPU reduces
    // sub-batch i (launches are asynchronous), and consecutive sub-batches
    // alternate between two streams so that the next persistent launch fills
    // the SMs the previous one's tail leaves idle.  Instances are taken
    // heaviest first (estimated from the precision alone: p x sum_m N_m x the
    // limb products per multiply-add), so that the longest instances start in
    // the first launch and the lighter ones fill the tails (4096 plane quintics
    // end to end on a GB300: 5.03 s in eight sub-batches of the input order,
    // 4.98 s in one, 3.83 s in eight heaviest-first).  Results go back in the
    // caller's order.
    const size_t S = count >= 2048 ? 8 : count >= 512 ? 4 : count >= 256 ? 2 : 1;
    std::vector<double> key(count, 0.0);
    zeta_options o = opt ? *opt : default_options();
    if (S > 1)
        parallel_for(count, ctx->threads, [&](size_t i) {
            Instance X;
            if (prepare_instance(&hs[i], &o, false, X) != ZETA_OK) return;
            uint32_t nsum = 0;
            for (uint32_t m = 0; m < X.n; m++) nsum += X.N[m];
            key[i] = (double)X.p * nsum * (X.q < ((uint64_t)1 << 56) ? 4.0 : 6.0);
        });
    std::vector<size_t> order(count);
    for (size_t i = 0; i < count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return key[x] > key[y]; });
    std::vector<zeta_hypersurface> hp(count);
    for (size_t i = 0; i < count; i++) hp[i] = hs[order[i]];
    std::vector<int64_t> Pp(2 * count * std::max<size_t>(stride, 1), 0);
    std::vector<zeta_stats> statp(per_instance ? count : 0);
    std::vector<zeta_batch_plan *> plans(S, nullptr);
    zeta_status st = ZETA_OK;
    // device-solved setups are begun for every sub-batch before the first launch: a solve queued
    // behind a running persistent launch would wait for it
    std::vector<Instance> begun;
    if (S > 1 && wants_device_setup(o, hp.data(), count)) {
        begun.resize(count);
        st = begin_on_device(ctx, hp.data(), count, o, begun.data(), nullptr);
    }
    for (size_t i = 0; i < S && !st; i++) {
        const size_t a = count * i / S, b = count * (i + 1) / S;
        st = batch_prepare_lane(ctx, hp.data() + a, b - a, opt, (int)(i & 1), &plans[i],
                                begun.empty() ? nullptr : begun.data() + a);
        if (!st) st = zeta_batch_run(ctx, plans[i]);
    }
    zeta_stats agg;
    std::memset(&agg, 0, sizeof(agg));
    for (size_t i = 0; i < S && !st; i++) {
        const size_t a = count * i / S, b = count * (i + 1) / S;
        zeta_stats part;
        st = zeta_batch_finish(ctx, plans[i], Pp.data() + 2 * a * stride, stride,
                               per_instance ? statp.data() + a : nullptr, &part);
        if (st) break;
        agg.chains += part.chains;
        agg.terms += part.terms;
        agg.chunks += part.chunks;
        agg.steps += part.steps;
        agg.column_steps += part.column_steps;
        agg.ms_host_setup += part.ms_host_setup;
        agg.ms_host_finish += part.ms_host_finish;
        agg.ms_kernel += part.ms_kernel;
        agg.kernel_launches += part.kernel_launches;
        agg.bytes_h2d += part.bytes_h2d;
        agg.bytes_d2h += part.bytes_d2h;
    }
    for (auto *P : plans) zeta_batch_release(P);
    if (st) return st;
    for (size_t i = 0; i < count; i++) {
        std::memcpy(P_out + 2 * order[i] * stride, Pp.data() + 2 * i * stride, sizeof(int64_t) * 2 * stride);
        if (per_instance) per_instance[order[i]] = statp[i];
    }
    if (total) *total = agg;
    return st;
}

zeta_status zeta_autotune(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count, const zeta_options *opt,
                          uint32_t sample, zeta_tuning *out) {
    if (!ctx || !hs || !count || !out) return ZETA_ERR_ARG;
    for (size_t i = 1; i < count; i++)
        if (hs[i].n != hs[0].n || hs[i].d != hs[0].d) return ZETA_ERR_ARG;
    // default sample: 16 instances per SM, so that every candidate runs in its steady state (a persistent
    // block takes several instances) rather than in the tail of a short queue
    const size_t want = std::min<size_t>(count, sample ? sample : (size_t)16 * engine_sm_count(ctx->engine));
    std::vector<zeta_hypersurface> pick(want);
    for (size_t i = 0; i < want; i++) pick[i] = hs[i * count / want];
    zeta_options base = opt ? *opt : default_options();
    zeta_tuning T;
    std::memset(&T, 0, sizeof(T));
    T.n = hs[0].n;
    T.d = hs[0].d;
    T.sample = (uint32_t)want;
    const uint32_t threads[4] = {0, 128, 256, 384};
    for (uint32_t th : threads) {
        T.cand_path[T.candidates] = ZETA_PATH_VECTOR;
        T.cand_threads[T.candidates++] = th;
    }
    T.cand_path[T.candidates] = ZETA_PATH_GEMM;  // dropped below if the instances are too large
    T.cand_threads[T.candidates++] = 0;
    std::vector<std::vector<int64_t>> results;
    size_t stride = 0;
    uint32_t kept = 0;
    for (uint32_t ci = 0; ci < T.candidates; ci++) {
        zeta_options o = base;
        o.path = (zeta_path)T.cand_path[ci];
        o.block_threads = T.cand_threads[ci];
        zeta_batch_plan *P = nullptr;
        zeta_status st = zeta_batch_prepare(ctx, pick.data(), pick.size(), &o, &P);
        if (st == ZETA_ERR_UNSUPPORTED && o.path == ZETA_PATH_GEMM) { ctx->error.clear(); continue; }
        if (st) return st;
        if (!stride)
            for (const Instance &X : P->inst) stride = std::max<size_t>(stride, (size_t)X.b + 1);
        st = zeta_batch_run(ctx, P);
        std::vector<int64_t> buf(2 * pick.size() * std::max<size_t>(stride, 1), 0);
        zeta_stats tot;
        if (!st) st = zeta_batch_finish(ctx, P, buf.data(), std::max<size_t>(stride, 1), nullptr, &tot);
        zeta_batch_release(P);
        if (st) return st;
        T.cand_path[kept] = T.cand_path[ci];
        T.cand_threads[kept] = T.cand_threads[ci];
        T.cand_ms[kept] = tot.kernel_launches ? tot.ms_kernel / (double)tot.kernel_launches : 0.0;
        kept++;
        results.push_back(std::move(buf));
    }
    T.candidates = kept;
    for (size_t i = 1; i < results.size(); i++)
        if (results[i] != results[0]) {
            ctx->error = "autotuner candidates disagree";
            return ZETA_ERR_INTERNAL;
        }
    for (uint32_t ci = 1; ci < kept; ci++)
        if (T.cand_ms[ci] < T.cand_ms[T.best]) T.best = ci;
    ctx->tuned[{T.n, T.d}] = T;
    *out = T;
    return ZETA_OK;
}

zeta_status zeta_selftest_wait(zeta_ctx *ctx, uint32_t limit_ms, double *waited_ms) {
    if (!ctx || limit_ms == 0 || limit_ms > 10000) return ZETA_ERR_ARG;
    return wait_selftest(limit_ms, waited_ms, ctx->error);
}

zeta_status zeta_horner_device(zeta_ctx *ctx, zeta_path path, uint32_t count, uint32_t s, uint32_t c,
                               const uint32_t *k, const uint64_t *A, const uint64_t *B, uint64_t *W,
                               const uint64_t *q) {
    if (!ctx || (count && (!k || !A || !B || !W || !q))) return ZETA_ERR_ARG;
    return engine_horner(ctx->engine, path, count, s, c, k, A, B, W, q, ctx->error);
}

zeta_status zeta_plan(const zeta_hypersurface *hs, const zeta_options *opt, zeta_plan_info *info, uint64_t *sec,
                      int32_t *chain_U, uint32_t *chain_terms, uint32_t *term_rc, uint64_t *term_coeff,
                      uint64_t *fin) {
    if (!hs) return ZETA_ERR_ARG;
    zeta_options o = opt ? *opt : default_options();
    Instance X;
    X.net.w = o.policy_weights;
    X.net.hidden = (int)o.policy_hidden;
    zeta_status st = prepare_instance(hs, &o, true, X);
    if (!st) st = schedule_policy(X, o.policy);
    if (st) return st;
    if (info) {
        info->plan_chunks = X.plan.chunks_played;
        info->plan_steps = X.plan.steps;
        info->plan_column_steps = X.plan.column_steps;
        info->plan_merges = X.plan.merges;
        info->plan_entries = X.plan.entries.size();
        info->plan_cap = X.plan.cap;
        info->b = X.b; info->s = X.s; info->nv = X.nv;
        info->sec_rows = X.sec_rows; info->sec_cols = X.sec_cols; info->h_rows = X.h_rows;
        info->r = X.r; info->M = X.M; info->q = X.q;
        info->nchains = X.chains.size(); info->nterms = X.terms.size();
        info->kappa = X.kappa; info->S_mask = X.Smask;
    }
    if (sec) std::memcpy(sec, X.sec.data(), sizeof(uint64_t) * X.sec.size());
    for (size_t c = 0; c < X.chains.size(); c++) {
        if (chain_U)
            for (uint32_t t = 0; t < X.nv; t++) chain_U[c * X.nv + t] = X.chains[c].U[t];
        if (chain_terms) { chain_terms[2 * c] = X.chains[c].term_begin; chain_terms[2 * c + 1] = X.chains[c].term_end; }
    }
    for (size_t t = 0; t < X.terms.size(); t++) {
        if (term_rc) { term_rc[2 * t] = X.terms[t].row; term_rc[2 * t + 1] = X.terms[t].col; }
        if (term_coeff) term_coeff[t] = X.terms[t].coeff;
    }
    if (fin) std::memcpy(fin, X.fin.data(), sizeof(uint64_t) * X.fin.size());
    return ZETA_OK;
}

zeta_status zeta_plan_device(zeta_ctx *ctx, const zeta_hypersurface *hs, const zeta_options *opt, uint64_t *sec,
                             uint64_t *fin, double *ms_device) {
    if (!ctx || !hs) return ZETA_ERR_ARG;
    if (ms_device) *ms_device = 0;
    if (!ctx->engine) { ctx->error = "no device engine"; return ZETA_ERR_DEVICE; }
    zeta_options o = opt ? *opt : default_options();
    Instance X;
    zeta_status st = prepare_instance(hs, &o, true, X, true);
    if (st) { ctx->error = X.error; return st; }
    std::vector<SolveJob *> jobs;
    std::vector<uint64_t> qs, ps;
    for (SolveJob &J : X.solves)
        if (J.R) {
            jobs.push_back(&J);
            qs.push_back(X.q);
            ps.push_back(X.p);
        }
    if ((st = engine_solve(ctx->engine, jobs, qs, ps, ctx->error, ms_device))) return st;
    for (SolveJob *J : jobs)
        if (!J->done) { ctx->error = "a right inverse is too wide for the device solve"; return ZETA_ERR_UNSUPPORTED; }
    if ((st = prepare_complete(X))) { ctx->error = X.error; return st; }
    if (sec) std::memcpy(sec, X.sec.data(), sizeof(uint64_t) * X.sec.size());
    if (fin) std::memcpy(fin, X.fin.data(), sizeof(uint64_t) * X.fin.size());
    return ZETA_OK;
}

zeta_status zeta_plan_tables(const zeta_hypersurface *hs, const zeta_options *opt, int32_t *monoS,
                             int32_t *secrow) {
    if (!hs) return ZETA_ERR_ARG;
    zeta_options o = opt ? *opt : default_options();
    Instance X;
    zeta_status st = prepare_instance(hs, &o, true, X);
    if (st) return st;
    if (monoS) std::memcpy(monoS, X.tab_monoS.data(), sizeof(int32_t) * X.tab_monoS.size());
    if (secrow) std::memcpy(secrow, X.tab_secrow.data(), sizeof(int32_t) * X.tab_secrow.size());
    return ZETA_OK;
}

zeta_status zeta_plan_moves(const zeta_hypersurface *hs, const zeta_options *opt, size_t *nphases, size_t *nentries,
                            size_t *nchunks, uint32_t *phase_begin, int32_t *entries, int32_t *chunks) {
    if (!hs || !nphases || !nentries || !nchunks) return ZETA_ERR_ARG;
    zeta_options o = opt ? *opt : default_options();
    Instance X;
    X.net.w = o.policy_weights;
    X.net.hidden = (int)o.policy_hidden;
    zeta_status st = prepare_instance(hs, &o, true, X);
    if (!st) st = schedule_policy(X, o.policy);
    if (st) return st;
    if (X.b > 32) return ZETA_ERR_UNSUPPORTED;  // `live` is exported as one 32-bit word
    const Plan &P = X.plan;
    const size_t nv = X.nv;
    *nphases = P.phase_begin.size() - 1;
    *nentries = P.entries.size();
    *nchunks = P.chunks.size();
    if (phase_begin) std::memcpy(phase_begin, P.phase_begin.data(), sizeof(uint32_t) * P.phase_begin.size());
    if (entries)
        for (size_t i = 0; i < P.entries.size(); i++) {
            const PlanEntry &e = P.entries[i];
            int32_t *o_ = entries + i * (nv + 7);
            for (size_t t = 0; t < nv; t++) o_[t] = e.U[t];
            o_[nv] = (int32_t)e.chunk_begin;
            o_[nv + 1] = (int32_t)e.chunk_end;
            o_[nv + 2] = e.arrival;
            o_[nv + 3] = e.start_chain;
            o_[nv + 4] = e.dest;
            o_[nv + 5] = (int32_t)e.flags;
            o_[nv + 6] = (int32_t)e.live;
        }
    if (chunks)
        for (size_t i = 0; i < P.chunks.size(); i++) {
            int32_t *o_ = chunks + i * (nv + 1);
            for (size_t t = 0; t < nv; t++) o_[t] = P.chunks[i].v[t];
            o_[nv] = P.chunks[i].k;
        }
    return ZETA_OK;
}

zeta_status zeta_policy_dataset(const zeta_hypersurface *hs, const zeta_options *opt, size_t *ngroups, size_t *ncand,
                                float *X, uint32_t *group_off, uint32_t *labels, int32_t *costs) {
    if (!hs || !ngroups || !ncand || !hs->coeffs) return ZETA_ERR_ARG;
    zeta_options o = opt ? *opt : default_options();
    // the rollouts are costly: the last instance's dataset is kept per host thread, so that the sizing call
    // and the filling call of the two-call protocol run them once
    struct Cached {
        std::vector<uint32_t> key;
        std::vector<float> feat;
        std::vector<uint32_t> goff, lab;
        std::vector<int32_t> cost;
    };
    static thread_local Cached cache;
    if (hs->n < 1 || hs->n > 7 || hs->d < 2 || hs->d > 12) return ZETA_ERR_UNSUPPORTED;
    size_t ncoef = 1;  // C(n + d, n)
    for (uint32_t i = 1; i <= hs->n; i++) ncoef = ncoef * (hs->d + i) / i;
    std::vector<uint32_t> key = {hs->n, hs->d, hs->p, o.r_override, o.S_mask};
    key.insert(key.end(), o.N_override, o.N_override + 8);
    key.insert(key.end(), hs->coeffs, hs->coeffs + ncoef);
    if (key != cache.key) {
        Instance I;
        zeta_status st = prepare_instance(hs, &o, true, I);
        if (st) return st;
        Cached c;
        st = policy_dataset(I, c.feat, c.goff, c.lab, c.cost);
        if (st) return st;
        c.key = key;
        cache = std::move(c);
    }
    *ngroups = cache.lab.size();
    *ncand = cache.cost.size();
    if (X) std::memcpy(X, cache.feat.data(), sizeof(float) * cache.feat.size());
    if (group_off) std::memcpy(group_off, cache.goff.data(), sizeof(uint32_t) * cache.goff.size());
    if (labels) std::memcpy(labels, cache.lab.data(), sizeof(uint32_t) * cache.lab.size());
    if (costs) std::memcpy(costs, cache.cost.data(), sizeof(int32_t) * cache.cost.size());
    return ZETA_OK;
}

zeta_status zeta_mlp_forward_host(uint32_t hidden, const float *params, const float *X, size_t n, float *scores) {
    if (!params || (n && (!X || !scores)) || hidden == 0 || hidden > 512) return ZETA_ERR_ARG;
    PolicyNet net;
    net.w = params;
    net.hidden = (int)hidden;
    for (size_t i = 0; i < n; i++) scores[i] = policy_score(net, X + i * kPolicyFeatures);
    return ZETA_OK;
}

zeta_status zeta_finish(const zeta_hypersurface *hs, const zeta_options *opt, const uint64_t *H, uint64_t *F_out,
                        uint64_t *Y_out, int64_t *P_out) {
    if (!hs || !H) return ZETA_ERR_ARG;
    zeta_options o = opt ? *opt : default_options();
    Instance X;
    zeta_status st = prepare_instance(hs, &o, true, X);
    if (st) return st;
    X.H.assign(H, H + (size_t)X.h_rows * X.b);
    st = finish_instance(X);
    if (st) return st;
    if (F_out) std::memcpy(F_out, X.F.data(), sizeof(uint64_t) * X.F.size());
    if (Y_out) std::memcpy(Y_out, X.Y.data(), sizeof(uint64_t) * X.Y.size());
    if (P_out)
        for (uint32_t i = 0; i <= X.b; i++) write_coeff(P_out + 2 * i, X.P[i]);
    return ZETA_OK;
}

}  // extern "C"
