"""GB300 controlled reduction: zeta functions of smooth hypersurfaces over F_p.

Thin Python binding of the C ABI in include/zeta.h (argument marshalling
only; every step of the computation runs in the native library and its CUDA
kernels).  The library must have been built (`paper_2602_24155_gb300.build`);
importing the package without it raises ImportError: there is no fallback.

    import paper_2602_24155_gb300 as z
    ctx = z.zeta_create(0)
    P, st = z.zeta_charpoly(ctx, (2, 4, 11, coeffs))
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libzeta.so")

POLICY = {"p_chunk": 0, "depth_first": 1, "var_by_var": 2, "learned": 3, "cover": 4}
POLICY_FEATURES = 18
PATH = {"vector": 0, "gemm": 1, "auto": 2}
PATH_NAME = {v: k for k, v in PATH.items()}

STATUS = {0: "ZETA_OK", 1: "ZETA_ERR_ARG", 2: "ZETA_ERR_NOT_SMOOTH", 3: "ZETA_ERR_UNSUPPORTED",
          4: "ZETA_ERR_PRECISION", 5: "ZETA_ERR_DEVICE", 6: "ZETA_ERR_TIMEOUT", 7: "ZETA_ERR_OOM",
          8: "ZETA_ERR_INTERNAL"}

EXPORTS = ["zeta_create", "zeta_destroy", "zeta_last_error", "zeta_query", "zeta_frobenius",
           "zeta_charpoly", "zeta_batch", "zeta_batch_prepare", "zeta_batch_run", "zeta_batch_finish",
           "zeta_batch_release", "zeta_horner_device", "zeta_horner_static", "zeta_plan", "zeta_finish",
           "zeta_mlp_param_count", "zeta_mlp_init", "zeta_mlp_forward", "zeta_mlp_grad", "zeta_mlp_train",
           "zeta_policy_dataset", "zeta_autotune", "zeta_selftest_wait", "zeta_plan_moves",
           "zeta_plan_tables", "zeta_mlp_forward_host", "zeta_plan_device"]
FLAG_Y_ONLY = 1
FLAG_HOST_SETUP = 2
FLAG_DEVICE_SETUP = 4
FLAG_WHOLE_GPU = 8
SETUP = {"auto": 0, "host": FLAG_HOST_SETUP, "device": FLAG_DEVICE_SETUP}


class ZetaError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s%s" % (STATUS.get(status, status), (": " + msg) if msg else ""))


class Hypersurface(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("d", ctypes.c_uint32), ("p", ctypes.c_uint32),
                ("coeffs", ctypes.POINTER(ctypes.c_uint32))]


class Options(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int), ("path", ctypes.c_int), ("r_override", ctypes.c_uint32),
                ("N_override", ctypes.c_uint32 * 8), ("flags", ctypes.c_uint32),
                ("policy_weights", ctypes.POINTER(ctypes.c_float)), ("policy_hidden", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("S_mask", ctypes.c_uint32)]


TUNE_MAX = 8


class Tuning(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("d", ctypes.c_uint32), ("sample", ctypes.c_uint32),
                ("candidates", ctypes.c_uint32), ("cand_path", ctypes.c_uint32 * TUNE_MAX),
                ("cand_threads", ctypes.c_uint32 * TUNE_MAX), ("cand_ms", ctypes.c_double * TUNE_MAX),
                ("best", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("b", ctypes.c_uint32), ("r", ctypes.c_uint32),
                ("M", ctypes.c_uint32), ("N", ctypes.c_uint32 * 8), ("s", ctypes.c_uint32),
                ("eps", ctypes.c_int32), ("chains", ctypes.c_uint64), ("terms", ctypes.c_uint64),
                ("chunks", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("column_steps", ctypes.c_uint64),
                ("ms_host_setup", ctypes.c_double), ("ms_device", ctypes.c_double),
                ("ms_host_finish", ctypes.c_double), ("ms_kernel", ctypes.c_double),
                ("kernel_launches", ctypes.c_uint64), ("bytes_h2d", ctypes.c_uint64),
                ("bytes_d2h", ctypes.c_uint64), ("ms_dev_start", ctypes.c_double), ("ms_dev_end", ctypes.c_double)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name == "N" else v
        return out


class PlanInfo(ctypes.Structure):
    _fields_ = [("b", ctypes.c_uint32), ("s", ctypes.c_uint32), ("nv", ctypes.c_uint32),
                ("sec_rows", ctypes.c_uint32), ("sec_cols", ctypes.c_uint32), ("h_rows", ctypes.c_uint32),
                ("r", ctypes.c_uint32), ("M", ctypes.c_uint32), ("q", ctypes.c_uint64),
                ("nchains", ctypes.c_uint64), ("nterms", ctypes.c_uint64),
                ("plan_chunks", ctypes.c_uint64), ("plan_steps", ctypes.c_uint64),
                ("plan_column_steps", ctypes.c_uint64), ("plan_merges", ctypes.c_uint64),
                ("plan_entries", ctypes.c_uint64), ("plan_cap", ctypes.c_uint64),
                ("kappa", ctypes.c_uint32), ("S_mask", ctypes.c_uint32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libzeta.so is not built: run `python -m paper_2602_24155_gb300.build` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    lib.zeta_create.argtypes = [P(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
    lib.zeta_destroy.argtypes = [ctypes.c_void_p]
    lib.zeta_last_error.argtypes = [ctypes.c_void_p]
    lib.zeta_last_error.restype = ctypes.c_char_p
    lib.zeta_query.argtypes = [P(Hypersurface), P(Options), P(ctypes.c_uint32), P(ctypes.c_uint32),
                               P(ctypes.c_uint32), P(ctypes.c_uint32)]
    lib.zeta_frobenius.argtypes = [ctypes.c_void_p, P(Hypersurface), P(Options), P(ctypes.c_uint64),
                                   P(ctypes.c_uint64), P(Stats)]
    lib.zeta_charpoly.argtypes = [ctypes.c_void_p, P(Hypersurface), P(Options), P(ctypes.c_int64), P(Stats)]
    lib.zeta_batch.argtypes = [ctypes.c_void_p, P(Hypersurface), ctypes.c_size_t, P(Options),
                               P(ctypes.c_int64), ctypes.c_size_t, P(Stats), P(Stats)]
    lib.zeta_horner_device.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
    lib.zeta_plan.argtypes = [P(Hypersurface), P(Options), P(PlanInfo), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.zeta_finish.argtypes = [P(Hypersurface), P(Options), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p]
    lib.zeta_horner_static.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
    lib.zeta_mlp_param_count.argtypes = [ctypes.c_uint32]
    lib.zeta_mlp_init.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p]
    lib.zeta_mlp_forward.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.c_void_p]
    lib.zeta_mlp_forward_host.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]
    lib.zeta_mlp_grad.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                  ctypes.c_void_p]
    lib.zeta_mlp_train.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_float, ctypes.c_void_p]
    lib.zeta_policy_dataset.argtypes = [P(Hypersurface), P(Options), P(ctypes.c_size_t), P(ctypes.c_size_t),
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.zeta_batch_prepare.argtypes = [ctypes.c_void_p, P(Hypersurface), ctypes.c_size_t, P(Options),
                                       P(ctypes.c_void_p)]
    lib.zeta_batch_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.zeta_batch_finish.argtypes = [ctypes.c_void_p, ctypes.c_void_p, P(ctypes.c_int64), ctypes.c_size_t,
                                      P(Stats), P(Stats)]
    lib.zeta_batch_release.argtypes = [ctypes.c_void_p]
    lib.zeta_plan_tables.argtypes = [P(Hypersurface), P(Options), ctypes.c_void_p, ctypes.c_void_p]
    lib.zeta_plan_device.argtypes = [ctypes.c_void_p, P(Hypersurface), P(Options), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double)]
    lib.zeta_plan_moves.argtypes = [P(Hypersurface), P(Options), P(ctypes.c_size_t), P(ctypes.c_size_t),
                                    P(ctypes.c_size_t), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.zeta_selftest_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]
    lib.zeta_autotune.argtypes = [ctypes.c_void_p, P(Hypersurface), ctypes.c_size_t, P(Options), ctypes.c_uint32,
                                  P(Tuning)]
    for name in EXPORTS:
        if name != "zeta_last_error":
            getattr(lib, name).restype = ctypes.c_int
    lib.zeta_mlp_param_count.restype = ctypes.c_size_t
    return lib


class _Lazy:
    """Loads libzeta.so on first use (so that the build step can import the package)."""
    _lib = None

    def __getattr__(self, name):
        if _Lazy._lib is None:
            _Lazy._lib = _load()
        return getattr(_Lazy._lib, name)


LIB = _Lazy()


def _options(policy="depth_first", path="vector", r=0, N=None, y_only=False, weights=None, hidden=0,
             block_threads=0, S=None, setup="auto", whole_gpu=False):
    """S: the index set of Prop. 3.3 as variable indices (None = the library's choice: {0..n} when
    d >= n + 1, else {n}).  setup: where batch calls solve the setup's right inverses ("auto",
    "host" or "device").  whole_gpu: run every instance on the whole-GPU executor (instances with
    C(dn, n) > 512 always are)."""
    o = Options()
    o.block_threads = block_threads
    o.S_mask = sum(1 << int(i) for i in set(S)) if S else 0
    o.flags = (FLAG_Y_ONLY if y_only else 0) | SETUP[setup] | (FLAG_WHOLE_GPU if whole_gpu else 0)
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float32)
        o.policy_weights = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        o.policy_hidden = hidden
        o._keep = w
    o.policy = POLICY[policy]
    o.path = PATH[path]
    o.r_override = r or 0
    if N:
        if isinstance(N, dict):
            for m, v in N.items():
                o.N_override[m - 1] = v
        else:
            for m in range(8):
                o.N_override[m] = N
    return o


def _hypersurface(spec):
    n, d, p, coeffs = spec
    arr = (ctypes.c_uint32 * len(coeffs))(*[int(c) for c in coeffs])
    hs = Hypersurface(n, d, p, arr)
    hs._keep = arr
    return hs


def _check(ctx, st):
    if st != 0:
        msg = LIB.zeta_last_error(ctx).decode() if ctx else ""
        raise ZetaError(st, msg)


def _coeff128(lo, hi):
    v = (int(hi) << 64) | (int(lo) & ((1 << 64) - 1))
    return v


def zeta_create(device=0, stream=None):
    ctx = ctypes.c_void_p()
    st = LIB.zeta_create(ctypes.byref(ctx), device, stream)
    if st:
        raise ZetaError(st, "zeta_create on device %d" % device)
    return ctx


def zeta_destroy(ctx):
    LIB.zeta_destroy(ctx)


def zeta_last_error(ctx):
    return LIB.zeta_last_error(ctx).decode()


def zeta_query(spec, **opt):
    hs = _hypersurface(spec)
    o = _options(**opt)
    b, r, M, s = (ctypes.c_uint32() for _ in range(4))
    st = LIB.zeta_query(ctypes.byref(hs), ctypes.byref(o), ctypes.byref(b), ctypes.byref(r),
                        ctypes.byref(M), ctypes.byref(s))
    _check(None, st)
    return b.value, r.value, M.value, s.value


def zeta_frobenius(ctx, spec, **opt):
    """Returns (F, Y, stats): F, Y as b x b uint64 arrays (see include/zeta.h)."""
    b, _, _, _ = zeta_query(spec, **opt)
    hs = _hypersurface(spec)
    o = _options(**opt)
    F = np.zeros((b, b), dtype=np.uint64)
    Y = np.zeros((b, b), dtype=np.uint64)
    stats = Stats()
    st = LIB.zeta_frobenius(ctx, ctypes.byref(hs), ctypes.byref(o),
                            F.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                            Y.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(stats))
    _check(ctx, st)
    return F, Y, stats.as_dict()


def zeta_charpoly(ctx, spec, **opt):
    """Returns (P, stats) with P the list a_0..a_b of Python ints."""
    b, _, _, _ = zeta_query(spec, **opt)
    hs = _hypersurface(spec)
    o = _options(**opt)
    buf = np.zeros(2 * (b + 1), dtype=np.int64)
    stats = Stats()
    st = LIB.zeta_charpoly(ctx, ctypes.byref(hs), ctypes.byref(o),
                           buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(stats))
    _check(ctx, st)
    return [_coeff128(buf[2 * i], buf[2 * i + 1]) for i in range(b + 1)], stats.as_dict()


def _spec_array(specs):
    count = len(specs)
    arr = (Hypersurface * max(count, 1))()
    keep = []
    for i, spec in enumerate(specs):
        hs = _hypersurface(spec)
        keep.append(hs._keep)
        arr[i] = hs
    arr._keep = keep
    return arr


def _stride(specs):
    return 1 + max(((d - 1) ** (n + 1) + (-1) ** (n + 1) * (d - 1)) // d for n, d, _, _ in specs)


def _unpack(buf, per, count, stride):
    out = []
    for i in range(count):
        if per[i].status != 0:
            out.append(None)
            continue
        b = per[i].b
        base = 2 * i * stride
        out.append([_coeff128(buf[base + 2 * t], buf[base + 2 * t + 1]) for t in range(b + 1)])
    return out


class BatchPlan:
    """Prepared batch (zeta_batch_prepare): inputs resident in device memory."""

    def __init__(self, ctx, specs, **opt):
        self.ctx = ctx
        self.count = len(specs)
        self.stride = _stride(specs) if specs else 1
        self._arr = _spec_array(specs)
        o = _options(**opt)
        self.handle = ctypes.c_void_p()
        _check(ctx, LIB.zeta_batch_prepare(ctx, self._arr, self.count, ctypes.byref(o), ctypes.byref(self.handle)))

    def run(self):
        """Enqueue the recurrence kernels on the context stream (asynchronous)."""
        _check(self.ctx, LIB.zeta_batch_run(self.ctx, self.handle))

    def finish(self):
        buf = np.zeros(2 * self.count * self.stride, dtype=np.int64)
        per = (Stats * max(self.count, 1))()
        total = Stats()
        _check(self.ctx, LIB.zeta_batch_finish(self.ctx, self.handle, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                               self.stride, per, ctypes.byref(total)))
        return _unpack(buf, per, self.count, self.stride), [per[i].as_dict() for i in range(self.count)], total.as_dict()

    def release(self):
        if self.handle:
            LIB.zeta_batch_release(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def zeta_batch_prepare(ctx, specs, **opt):
    return BatchPlan(ctx, specs, **opt)


def zeta_batch_run(ctx, plan):
    plan.run()


def zeta_batch_finish(ctx, plan):
    return plan.finish()


def zeta_batch_release(plan):
    plan.release()


def zeta_batch(ctx, specs, stride=None, **opt):
    """Returns (list of P or None, per-instance stats, total stats)."""
    count = len(specs)
    arr = _spec_array(specs)
    if stride is None:
        stride = _stride(specs)
    o = _options(**opt)
    buf = np.zeros(2 * count * stride, dtype=np.int64)
    per = (Stats * max(count, 1))()
    total = Stats()
    st = LIB.zeta_batch(ctx, arr, count, ctypes.byref(o), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                        stride, per, ctypes.byref(total))
    _check(ctx, st)
    return _unpack(buf, per, count, stride), [per[i].as_dict() for i in range(count)], total.as_dict()


def zeta_horner_device(ctx, path, count, s, c, k, A, B, W, q):
    """Kernel-level Algorithm 2 on device tensors (torch CUDA tensors or raw pointers)."""
    def ptr(x):
        return x if isinstance(x, int) else x.data_ptr()
    st = LIB.zeta_horner_device(ctx, PATH[path] if isinstance(path, str) else path, count, s, c,
                                ptr(k), ptr(A), ptr(B), ptr(W), ptr(q))
    _check(ctx, st)


def zeta_plan(spec, **opt):
    """Host setup of one instance; returns a dict of numpy arrays (see include/zeta.h)."""
    hs = _hypersurface(spec)
    o = _options(**opt)
    info = PlanInfo()
    _check(None, LIB.zeta_plan(ctypes.byref(hs), ctypes.byref(o), ctypes.byref(info), None, None, None,
                               None, None, None))
    sec = np.zeros((info.sec_rows, info.sec_cols), dtype=np.uint64)
    U = np.zeros((info.nchains, info.nv), dtype=np.int32)
    ct = np.zeros((info.nchains, 2), dtype=np.uint32)
    rc = np.zeros((info.nterms, 2), dtype=np.uint32)
    co = np.zeros(info.nterms, dtype=np.uint64)
    fin = np.zeros((info.b, info.h_rows), dtype=np.uint64)
    _check(None, LIB.zeta_plan(ctypes.byref(hs), ctypes.byref(o), ctypes.byref(info), sec.ctypes.data,
                               U.ctypes.data, ct.ctypes.data, rc.ctypes.data, co.ctypes.data, fin.ctypes.data))
    return dict(b=info.b, s=info.s, nv=info.nv, r=info.r, M=info.M, q=info.q, h_rows=info.h_rows,
                kappa=info.kappa, S=tuple(i for i in range(info.nv) if (info.S_mask >> i) & 1),
                sec=sec, U=U, chain_terms=ct, term_rc=rc, term_coeff=co, fin=fin,
                game=dict(chunks=info.plan_chunks, steps=info.plan_steps, column_steps=info.plan_column_steps,
                          merges=info.plan_merges, entries=info.plan_entries, cap=info.plan_cap))


def plan_sizes(spec, **opt):
    """(b, sec_rows, sec_cols, h_rows) of zeta_plan's outputs, from n, d, S and zeta_query alone (no setup):
    the section has (n+1) C(kappa-d+1+n, n) rows and C(kappa+n, n) columns, kappa = (n+1)(d-1)+1-|S|, and the
    final map C(dn-1, n) columns."""
    from math import comb
    n, d, _, _ = spec
    S = opt.get("S")
    size_S = len(set(S)) if S else (n + 1 if d >= n + 1 else 1)
    kappa = (n + 1) * (d - 1) + 1 - size_S
    b = zeta_query(spec, **opt)[0]
    return b, (n + 1) * comb(kappa - d + 1 + n, n), comb(kappa + n, n), comb(d * n - 1, n)


def zeta_plan_device(ctx, spec, **opt):
    """zeta_plan's section and final reduction map with the right inverses solved on the device (any C(dn, n) up to
    4096).  Returns (sec, fin, kernel ms)."""
    hs = _hypersurface(spec)
    o = _options(**opt)
    b, rows, cols, h_rows = plan_sizes(spec, **opt)
    sec = np.zeros((rows, cols), dtype=np.uint64)
    fin = np.zeros((b, h_rows), dtype=np.uint64)
    ms = ctypes.c_double(0)
    _check(ctx, LIB.zeta_plan_device(ctx, ctypes.byref(hs), ctypes.byref(o), sec.ctypes.data, fin.ctypes.data,
                                     ctypes.byref(ms)))
    return sec, fin, ms.value


def zeta_finish(spec, H, **opt):
    """Normalisation and P(T) from numerators H (h_rows x b uint64).  Returns (F, Y, P)."""
    b, _, _, _ = zeta_query(spec, **opt)
    hs = _hypersurface(spec)
    o = _options(**opt)
    H = np.ascontiguousarray(np.asarray(H, dtype=np.uint64))
    F = np.zeros((b, b), dtype=np.uint64)
    Y = np.zeros((b, b), dtype=np.uint64)
    buf = np.zeros(2 * (b + 1), dtype=np.int64)
    _check(None, LIB.zeta_finish(ctypes.byref(hs), ctypes.byref(o), H.ctypes.data, F.ctypes.data,
                                 Y.ctypes.data, buf.ctypes.data))
    return F, Y, [_coeff128(buf[2 * i], buf[2 * i + 1]) for i in range(b + 1)]


def zeta_horner_static(stream, count, s, c, k, A, B, W, q):
    """Allocation-free kernel-level Algorithm 2 on the current device (see include/zeta.h)."""
    def ptr(x):
        return x if isinstance(x, int) else x.data_ptr()
    st = LIB.zeta_horner_static(stream, count, s, c, ptr(k), ptr(A), ptr(B), ptr(W), ptr(q))
    _check(None, st)


# ---------------------------------------------------------------------------
# Learned policy: network and training data (include/zeta.h)
# ---------------------------------------------------------------------------
def zeta_mlp_param_count(hidden):
    return LIB.zeta_mlp_param_count(hidden)


def zeta_mlp_init(hidden, seed):
    w = np.zeros(zeta_mlp_param_count(hidden), dtype=np.float32)
    _check(None, LIB.zeta_mlp_init(hidden, seed, w.ctypes.data))
    return w


def zeta_mlp_forward(ctx, hidden, params, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    params = np.ascontiguousarray(params, dtype=np.float32)
    out = np.zeros(X.shape[0], dtype=np.float32)
    _check(ctx, LIB.zeta_mlp_forward(ctx, hidden, params.ctypes.data, X.ctypes.data, X.shape[0], out.ctypes.data))
    return out


def zeta_mlp_forward_host(hidden, params, X):
    """Scores computed by the host forward pass the scheduler uses."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    params = np.ascontiguousarray(params, dtype=np.float32)
    out = np.zeros(X.shape[0], dtype=np.float32)
    _check(None, LIB.zeta_mlp_forward_host(hidden, params.ctypes.data, X.ctypes.data, X.shape[0], out.ctypes.data))
    return out


def zeta_mlp_grad(ctx, hidden, params, X, group_off, labels):
    X = np.ascontiguousarray(X, dtype=np.float32)
    params = np.ascontiguousarray(params, dtype=np.float32)
    go = np.ascontiguousarray(group_off, dtype=np.uint32)
    lab = np.ascontiguousarray(labels, dtype=np.uint32)
    grad = np.zeros_like(params)
    loss = np.zeros(1, dtype=np.float32)
    _check(ctx, LIB.zeta_mlp_grad(ctx, hidden, params.ctypes.data, X.ctypes.data, go.ctypes.data, lab.ctypes.data,
                                  len(lab), grad.ctypes.data, loss.ctypes.data))
    return grad, float(loss[0])


def zeta_mlp_train(ctx, hidden, params, X, group_off, labels, epochs, batch_groups, lr):
    X = np.ascontiguousarray(X, dtype=np.float32)
    p = np.array(params, dtype=np.float32, copy=True)
    go = np.ascontiguousarray(group_off, dtype=np.uint32)
    lab = np.ascontiguousarray(labels, dtype=np.uint32)
    loss = np.zeros(1, dtype=np.float32)
    _check(ctx, LIB.zeta_mlp_train(ctx, hidden, p.ctypes.data, X.ctypes.data, go.ctypes.data, lab.ctypes.data,
                                   len(lab), epochs, batch_groups, lr, loss.ctypes.data))
    return p, float(loss[0])


def zeta_policy_dataset(spec, **opt):
    """Training decisions of one instance: (X, group_off, labels, costs)."""
    hs = _hypersurface(spec)
    o = _options(**opt)
    ng, nc = ctypes.c_size_t(), ctypes.c_size_t()
    _check(None, LIB.zeta_policy_dataset(ctypes.byref(hs), ctypes.byref(o), ctypes.byref(ng), ctypes.byref(nc),
                                         None, None, None, None))
    X = np.zeros((nc.value, POLICY_FEATURES), dtype=np.float32)
    go = np.zeros(ng.value + 1, dtype=np.uint32)
    lab = np.zeros(ng.value, dtype=np.uint32)
    cost = np.zeros(nc.value, dtype=np.int32)
    _check(None, LIB.zeta_policy_dataset(ctypes.byref(hs), ctypes.byref(o), ctypes.byref(ng), ctypes.byref(nc),
                                         X.ctypes.data, go.ctypes.data, lab.ctypes.data, cost.ctypes.data))
    return X, go, lab, cost


def zeta_autotune(ctx, specs, sample=0, **opt):
    """Times the candidate launch configurations on a sample of `specs` (all of one (n, d)) and records the
    fastest in the context for path="auto".  Returns {"best": {...}, "candidates": [...], "sample": m}."""
    arr = _spec_array(specs)
    o = _options(**opt)
    t = Tuning()
    _check(ctx, LIB.zeta_autotune(ctx, arr, len(specs), ctypes.byref(o), sample, ctypes.byref(t)))
    cands = [{"path": PATH_NAME[t.cand_path[i]], "block_threads": t.cand_threads[i], "ms": t.cand_ms[i]}
             for i in range(t.candidates)]
    return {"n": t.n, "d": t.d, "sample": t.sample, "candidates": cands, "best": cands[t.best]}


def zeta_selftest_wait(ctx, limit_ms):
    """Runs the bounded-wait self-test; returns (status, waited_ms) without raising (ZETA_ERR_TIMEOUT = 6 expected)."""
    w = ctypes.c_double(0.0)
    st = LIB.zeta_selftest_wait(ctx, limit_ms, ctypes.byref(w))
    return st, w.value


def zeta_plan_tables(spec, **opt):
    """The index tables the device's step-matrix generation reads (host only): dict with 'monoS'
    (s x nv, exponents mu + 1 - 1_S) and 'secrow' (nv x s, rows of the section or -1)."""
    hs = _hypersurface(spec)
    o = _options(**opt)
    info = PlanInfo()
    _check(None, LIB.zeta_plan(ctypes.byref(hs), ctypes.byref(o), ctypes.byref(info), None, None, None,
                               None, None, None))
    monoS = np.zeros((info.s, info.nv), dtype=np.int32)
    secrow = np.zeros((info.nv, info.s), dtype=np.int32)
    _check(None, LIB.zeta_plan_tables(ctypes.byref(hs), ctypes.byref(o), monoS.ctypes.data, secrow.ctypes.data))
    return {"monoS": monoS, "secrow": secrow}


def zeta_plan_moves(spec, **opt):
    """The scheduled moves of one instance (host only): dict with 'phase_begin', 'entries' (rows of
    U[nv], chunk_begin, chunk_end, arrival, start_chain, dest, flags, live) and 'chunks' (rows of v[nv], k)."""
    hs = _hypersurface(spec)
    o = _options(**opt)
    npha, nent, nchk = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(None, LIB.zeta_plan_moves(ctypes.byref(hs), ctypes.byref(o), ctypes.byref(npha), ctypes.byref(nent),
                                     ctypes.byref(nchk), None, None, None))
    nv = spec[0] + 1
    ph = np.zeros(npha.value + 1, dtype=np.uint32)
    ent = np.zeros((nent.value, nv + 7), dtype=np.int32)
    chk = np.zeros((max(nchk.value, 1), nv + 1), dtype=np.int32)
    _check(None, LIB.zeta_plan_moves(ctypes.byref(hs), ctypes.byref(o), ctypes.byref(npha), ctypes.byref(nent),
                                     ctypes.byref(nchk), ph.ctypes.data, ent.ctypes.data, chk.ctypes.data))
    return {"phase_begin": ph, "entries": ent, "chunks": chk[:nchk.value]}
