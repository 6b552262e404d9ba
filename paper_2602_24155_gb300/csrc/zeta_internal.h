// Internal interfaces between the host setup (zeta_host.cpp) and the CUDA
// kernels (zeta_kernels.cu).  Not part of the public ABI.
#pragma once
#include <array>
#include <cstdint>
#include <functional>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/zeta.h"

namespace zeta {

typedef unsigned __int128 u128;
typedef __int128 i128;

constexpr int kMaxVars = 8;

// ---------------------------------------------------------------------------
// Per-instance data prepared on the host (Prop. 2.1, Alg. 1, Prop. 3.3).
// ---------------------------------------------------------------------------
struct Term {
    uint32_t row;    // index of J in Homog_{dn-n} (descending lex)
    uint32_t col;    // basis column
    uint64_t coeff;  // mod q
};

struct Chain {
    int32_t U[kMaxVars];     // start exponent (pole order (|U|-n)/d + n)
    uint32_t term_begin, term_end;
    uint64_t work;           // estimated steps * s^2 * b
};

// A reduction plan: the game of Sec. 3.4 played on the host (integer-only),
// executed on the device.  Phases run in order; within a phase every entry is
// one term: its W block is formed from an arrival block (the merged results
// of the previous phase that landed on this exponent) and/or the start terms
// of one chain, then reduced by its chunk list (move 1: k steps in direction
// v, Sec. 3.4), then merged into a block of the next phase (move 2) or, at
// pole order n, accumulated into the numerators H.
struct PlanChunk {
    int8_t v[kMaxVars];
    int32_t k;
};

struct PlanEntry {
    int32_t U[kMaxVars];         // exponent at the start of the phase
    uint32_t chunk_begin, chunk_end;
    int32_t arrival;             // block of the current phase buffer, or -1
    int32_t start_chain;         // chain whose start terms join here, or -1
    int32_t dest;                // block of the next phase buffer, -1: pole order n reached
    uint32_t flags;              // bit 0: first contribution to dest (store, not add)
    uint64_t live;               // basis columns carried (bit mask, b <= 64)
};

struct Plan {
    std::vector<PlanEntry> entries;
    std::vector<PlanChunk> chunks;
    std::vector<uint32_t> phase_begin;  // nphases + 1 offsets into entries
    uint32_t cap = 0;                   // blocks per phase buffer
    uint64_t chunks_played = 0, steps = 0, column_steps = 0, merges = 0, work = 0;
};

// Learned direction policy (zeta_learn.cpp).
constexpr int kPolicyFeatures = 18;
struct PolicyNet {
    const float *w = nullptr;  // W1 (F x H), b1 (H), W2 (H x H), b2 (H), w3 (H), b3 (1)
    int hidden = 0;
};

// One right inverse over Z/q (Prop. 3.3 section; the final reduction's levels, Sec. 3.3 step (2)):
// A (R x C, full row rank mod p) in, X (C x R, A X = I) out, both in Montgomery form (R = 2^64).
// Solved on the host (right_inverse) or on the device (engine_solve); both run Gauss-Jordan
// with unit pivots, columns in order, the first unit row as pivot, so both give the same X.
struct SolveJob {
    int R = 0, C = 0;
    std::vector<uint64_t> A;
    std::vector<uint64_t> X;
    bool done = false, ok = false;
};

struct Instance {
    // input
    uint32_t n = 0, d = 0, p = 0, nv = 0;
    std::vector<uint32_t> coeffs;
    // sizes
    uint32_t b = 0, s = 0;       // basis size, |Homog_{dn-n}|
    uint32_t kappa = 0;          // (n+1)(d-1)+1-|S|; (n+1)(d-2)+1 for S = {0..n}
    uint32_t Smask = 0;          // index set S of Prop. 3.3 (bit i = i in S)
    uint32_t base = 0;           // |S| - 1: |u| of a term at pole order n
    uint32_t sec_rows = 0, sec_cols = 0;
    uint32_t h_rows = 0;         // |Homog_{dn-n-1}|
    // precision
    uint32_t r = 0, M = 0;             // r = max_m r_m
    uint32_t rm[kMaxVars] = {0};       // r_m, m = 1..n (index m-1)
    uint32_t N[kMaxVars] = {0};
    uint64_t q = 0;
    std::vector<uint32_t> pole;  // pole order of each basis element
    std::vector<std::vector<int>> basis_exp;
    // controlled reduction data
    std::vector<uint64_t> sec;   // sec_rows x sec_cols, Sec[(i,nu), gamma]
    std::vector<Chain> chains;
    std::vector<Term> terms;
    std::vector<uint64_t> fin;   // b x h_rows final reduction map mod q
    // index tables of the device's step-matrix generation (zeta_plan_tables)
    std::vector<int32_t> tab_monoS;   // s x nv: mu + 1 - 1_S
    std::vector<int32_t> tab_secrow;  // nv x s: row (i, omega - 1_S + e_i) of sec, or -1
    // right inverses of the reduction build: [0] the section, [m] the final reduction at pole order m
    std::vector<SolveJob> solves;
    bool solves_pending = false;      // prepare_instance stopped before using them (prepare_complete resumes)
    Plan plan;
    PolicyNet net;              // learned policy (ZETA_POLICY_LEARNED)
    // per level t: exponent -> terms reaching it in the reference game (the cover game with Algorithm 3), and
    // for each basis column the number of those terms that carry it
    std::vector<std::unordered_map<uint64_t, int>> ref_contrib;
    std::vector<std::unordered_map<uint64_t, std::array<uint16_t, 64>>> ref_cols;
    // columns carried by the term whose chunk direction is being chosen (set by the scheduler before it asks)
    mutable uint64_t cur_live = 0;
    // ZETA_POLICY_COVER with a decision hook: the hook chooses the direction of every chunk decision
    // (U, steps left in the p-chunk, level t); false = Algorithm 3 (training-data rollouts)
    std::function<bool(const int32_t *U, int left, int t, int *v)> hook;
    // results
    std::vector<uint64_t> H;     // h_rows x b accumulated numerators mod q
    std::vector<uint64_t> Y;     // b x b
    std::vector<uint64_t> F;     // b x b
    std::vector<i128> P;         // b+1
    int eps = 0;
    zeta_status status = ZETA_OK;
    std::string error;
    uint64_t nterms = 0, steps = 0, column_steps = 0, chunks = 0;
    double ms_setup = 0, ms_finish = 0;
    double ms_dev_start = 0, ms_dev_end = 0;  // instance start and end in its launch (device clock)
};

// Host-side steps (zeta_host.cpp)
// defer_solves: stop once the right inverses' matrices are built (X.solves, X.solves_pending), so that
// they can be solved together on the device; prepare_complete solves what is left on the host and
// finishes the reduction data.
zeta_status prepare_instance(const zeta_hypersurface *hs, const zeta_options *opt,
                             bool build_reduction, Instance &X, bool defer_solves = false);
zeta_status prepare_complete(Instance &X);
zeta_status finish_instance(Instance &X);
// Plays the policy on the start chains of X and fills X.plan (zeta_policy.cpp).
zeta_status validate_plan(Instance &X);
zeta_status schedule_policy(Instance &X, zeta_policy policy);

size_t policy_param_count(int hidden);
// Chooses the direction of a chunk of the p-chunk of the term at U (level t of tmax,
// `left` steps left); false when no network is set or only one direction is legal.
bool learned_direction(const Instance &X, const int32_t *U, int left, int t, int tmax, int *v);
// Training decisions labelled by rollouts of the cover game (see zeta_learn.cpp).
constexpr int kDatasetDecisions = 128;  // decisions sampled per instance
constexpr int kChunkCost = 10;          // setup of one chunk in column steps (measured)
zeta_status policy_dataset(Instance &X, std::vector<float> &feat, std::vector<uint32_t> &group_off,
                           std::vector<uint32_t> &labels, std::vector<int32_t> &costs);
// Host copy of the network's forward pass, used by the scheduler (zeta_mlp_forward_host).
float policy_score(const PolicyNet &net, const float *x);
// Plays the reference game (the cover game with Algorithm 3) and records, per level, how many terms reach each
// exponent and which columns they carry.
zeta_status reference_contributions(Instance &X);
zeta_status finish_y_only(Instance &X);  // Y = Fin * H only

// Device engine (zeta_kernels.cu): runs the recurrence for every chain of
// every instance and fills X.H.  `policy` selects the reduction policy.
struct DeviceEngine;
DeviceEngine *engine_create(int device, void *stream, std::string &err);
void engine_destroy(DeviceEngine *e);
int engine_sm_count(const DeviceEngine *e);
// Bounded-wait self-test on the current device (zeta_selftest.cu).
zeta_status wait_selftest(uint32_t limit_ms, double *waited_ms, std::string &err);
zeta_status engine_run(DeviceEngine *e, std::vector<Instance *> &batch, zeta_policy policy, zeta_path path,
                       uint32_t block_threads, std::string &err, double *ms_device);
// The same in three phases: upload (inputs become resident in device
// memory), launch (kernels only, asynchronous on the engine's stream),
// collect (synchronise and read H back).
struct DeviceBatch;
// lane 0: the engine's stream; lane 1: a second, non-blocking stream, so that
// consecutive batches overlap (the next launch's blocks take the SMs the
// previous launch's tail leaves idle).
zeta_status engine_prepare(DeviceEngine *e, std::vector<Instance *> &batch, zeta_policy policy, zeta_path path,
                           uint32_t block_threads, int lane, DeviceBatch **out, std::string &err);
zeta_status engine_launch(DeviceEngine *e, DeviceBatch *B, std::string &err);
zeta_status engine_collect(DeviceEngine *e, DeviceBatch *B, std::string &err);
void engine_release(DeviceBatch *B);
void engine_batch_timing(const DeviceBatch *B, double *ms_kernel, uint64_t *launches, uint64_t *h2d, uint64_t *d2h);
zeta_status engine_horner(DeviceEngine *e, zeta_path path, uint32_t count, uint32_t s, uint32_t c,
                          const uint32_t *k, const uint64_t *A, const uint64_t *B, uint64_t *W,
                          const uint64_t *q, std::string &err);
// Solves the jobs on the device (zeta_setup.cuh), each modulo qs[t] with unit test mod ps[t];
// sets done, ok (full row rank) and X.  Jobs too wide for the kernel's shared memory are left undone.
// Runs the instances' plans on the whole-GPU executor (zeta_large.cuh) and fills their H (s <= 4096, b <= 64,
// q < 2^56): s > 512 one at a time; smaller ones up to eight at a time on lanes of their own.  ms_device: CUDA-event
// time of the former plus the elapsed time of the latter.  Each instance's start and completion go to
// ms_dev_start / ms_dev_end as host-clock milliseconds after t_ref_ms (steady clock).
zeta_status engine_run_large(DeviceEngine *e, std::vector<Instance *> &xs, std::string &err, double *ms_device,
                             uint64_t *launches, double t_ref_ms);
zeta_status engine_solve(DeviceEngine *e, const std::vector<SolveJob *> &jobs, const std::vector<uint64_t> &qs,
                         const std::vector<uint64_t> &ps, std::string &err, double *ms_device);

}  // namespace zeta
