"""Thin Python binding of libdetlsh.so (include/detlsh.h).

Argument marshalling only: every step of DET-LSH runs in the library's CUDA
kernels.  Functions keep the C-ABI names.  Arrays may be numpy (host) or torch
CUDA tensors (device); outputs follow the inputs' placement.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdetlsh.so")

DETLSH_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "NONFINITE_INPUT", -3: "OOM", -4: "CUDA",
          -5: "CAPACITY", -6: "NO_DEVICE", -7: "SCRATCH_LIMIT",
          -8: "TIMEOUT", -9: "IO", -10: "FORMAT"}
BOX_PREFIX, BOX_TIGHT = 0, 1
PREC_FP32, PREC_BF16_REFINE = 0, 1
RMIN_MAGIC, RMIN_FIXED, RMIN_CONTINUOUS = 0, 1, 2
ENC_DYNAMIC, ENC_STATIC = 0, 1


class DetlshError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, status_string(status), status))


class BuildParams(C.Structure):
    _fields_ = [("L", C.c_int32), ("K", C.c_int32), ("N_r", C.c_int32), ("max_size", C.c_int32),
                ("seed", C.c_uint64), ("sample_frac", C.c_double), ("box_mode", C.c_int32),
                ("keep_bf16", C.c_int32), ("keep_projections", C.c_int32),
                ("encoding", C.c_int32), ("tree_group", C.c_int32)]


class QueryParams(C.Structure):
    _fields_ = [("beta", C.c_double), ("c", C.c_double), ("precision", C.c_int32),
                ("rerank_mult", C.c_int32), ("rmin_policy", C.c_int32), ("r_min", C.c_double),
                ("per_tree", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("L", C.c_int32), ("K", C.c_int32),
                ("N_r", C.c_int32), ("max_size", C.c_int32), ("box_mode", C.c_int32),
                ("has_bf16", C.c_int32), ("sample_size", C.c_int64),
                ("num_leaves", C.c_int64 * 16), ("max_leaf_size", C.c_int64),
                ("eps2", C.c_double), ("device_bytes", C.c_int64),
                ("projection_fallbacks", C.c_int64), ("encoding", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("query_ctas_per_sm", C.c_int32), ("expand_runs", C.c_int32),
                ("visit_chunk", C.c_int32), ("top_hull_min", C.c_int32),
                ("hash_kb", C.c_int32), ("query_scratch_mb", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Timings(C.Structure):
    _fields_ = [("build_ms", C.c_float), ("sample_ms", C.c_float),
                ("breakpoints_ms", C.c_float), ("encode_ms", C.c_float),
                ("trees_ms", C.c_float), ("query_ms", C.c_float),
                ("query_project_ms", C.c_float), ("query_kernel_ms", C.c_float),
                ("build_launches", C.c_int64), ("query_launches", C.c_int64),
                ("query_count", C.c_int64), ("query_candidates", C.c_int64),
                ("query_leaves", C.c_int64), ("query_blocks", C.c_int64),
                ("query_points_visited", C.c_int64), ("query_reranked", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# (name, restype, argtypes) of every entry point declared in include/detlsh.h
_P, _I32, _I64, _F32P, _F64 = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_double
SIGNATURES = [
    ("detlsh_default_build_params", C.c_int, [C.POINTER(BuildParams)]),
    ("detlsh_default_query_params", C.c_int, [C.POINTER(QueryParams)]),
    ("detlsh_build", C.c_int, [_P, _I64, _I32, _I32, _I32, _I32, C.c_uint64, C.POINTER(_P)]),
    ("detlsh_build_ex", C.c_int, [_P, _I64, _I32, C.POINTER(BuildParams), _P, C.POINTER(_P)]),
    ("detlsh_query", C.c_int, [_P, _P, _I64, _I32, _F64, _P, _P]),
    ("detlsh_query_ex", C.c_int, [_P, _P, _I64, _P, _I32, C.POINTER(QueryParams), _P, _P, _P]),
    ("detlsh_query_noalloc", C.c_int, [_P, _P, _I64, _I32, C.POINTER(QueryParams), _P, _P, _P]),
    ("detlsh_save", C.c_int, [_P, C.c_char_p, _P]),
    ("detlsh_load", C.c_int, [C.c_char_p, _P, C.POINTER(_P)]),
    ("detlsh_free", C.c_int, [_P]),
    ("detlsh_get_tuning", C.c_int, [_P, C.POINTER(Tuning)]),
    ("detlsh_set_tuning", C.c_int, [_P, C.POINTER(Tuning)]),
    ("detlsh_autotune", C.c_int, [_P, _P, _I64, _I32, C.POINTER(QueryParams), C.c_char_p, _P,
                                  C.POINTER(Tuning), C.POINTER(C.c_int32)]),
    ("detlsh_status_string", C.c_char_p, [C.c_int]),
    ("detlsh_get_info", C.c_int, [_P, C.POINTER(Info)]),
    ("detlsh_get_projection_matrix", C.c_int, [_P, _P]),
    ("detlsh_get_sample", C.c_int, [_P, _P]),
    ("detlsh_get_breakpoints", C.c_int, [_P, _P]),
    ("detlsh_get_codes", C.c_int, [_P, _P]),
    ("detlsh_get_projections", C.c_int, [_P, _P]),
    ("detlsh_get_tree", C.c_int, [_P, _I32, _P, _P, _P, _P, _P, _P]),
    ("detlsh_get_level_table", C.c_int, [_P, _F64, _P]),
    ("detlsh_get_timings", C.c_int, [_P, C.POINTER(Timings)]),
    ("detlsh_project", C.c_int, [_P, _P, _I64, _P, _P]),
    ("detlsh_query_candidates", C.c_int, [_P, _P, _I64, _I32, C.POINTER(QueryParams), _I64,
                                          _P, _P, _P, _P]),
    ("detlsh_query_reserve", C.c_int, [_P, _I64, _I32, C.POINTER(QueryParams)]),
    ("detlsh_query_async", C.c_int, [_P, _P, _I64, _P, _I32, _P, _P, _P, _P]),
    ("detlsh_rc_ann", C.c_int, [_P, _P, _I64, _F64, _F64, _F64, _I32, _P, _P, _P, _P, _I64, _P,
                                _P]),
]


def lib():
    """Load libdetlsh.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libdetlsh.so is missing (%s): build it with "
                              "paper_2603_24920_gb300.build_ext.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(s):
    return lib().detlsh_status_string(s).decode()


def _check(s, what):
    if s != DETLSH_OK:
        raise DetlshError(s, what)


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data)


def _is_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def detlsh_default_build_params():
    p = BuildParams()
    _check(lib().detlsh_default_build_params(C.byref(p)), "detlsh_default_build_params")
    return p


def detlsh_default_query_params():
    p = QueryParams()
    _check(lib().detlsh_default_query_params(C.byref(p)), "detlsh_default_query_params")
    return p


def detlsh_build(data, L=4, K=16, N_r=256, seed=0, **kw):
    """detlsh_build_ex with defaults; data: (n, d) float32 numpy or CUDA tensor."""
    n, d = data.shape
    p = detlsh_default_build_params()
    p.L, p.K, p.N_r, p.seed = L, K, N_r, seed
    for k, v in kw.items():
        if k == "stream":
            continue
        setattr(p, k, v)
    h = C.c_void_p()
    _check(lib().detlsh_build_ex(_ptr(data), n, d, C.byref(p), _stream_ptr(kw.get("stream")),
                                 C.byref(h)), "detlsh_build_ex")
    return h


def detlsh_save(h, path, stream=None):
    """Write the index to an index file at path (str or os.PathLike)."""
    _check(lib().detlsh_save(h, os.fsencode(path), _stream_ptr(stream)), "detlsh_save")


def detlsh_load(path, stream=None):
    """Read an index file into a new index on the current device."""
    h = C.c_void_p()
    _check(lib().detlsh_load(os.fsencode(path), _stream_ptr(stream), C.byref(h)), "detlsh_load")
    return h


def detlsh_get_tuning(h):
    t = Tuning()
    _check(lib().detlsh_get_tuning(h, C.byref(t)), "detlsh_get_tuning")
    return t


def detlsh_set_tuning(h, query_ctas_per_sm=0, expand_runs=4, visit_chunk=512, top_hull_min=1024,
                      hash_kb=0, query_scratch_mb=0):
    t = Tuning(query_ctas_per_sm, expand_runs, visit_chunk, top_hull_min, hash_kb, query_scratch_mb)
    _check(lib().detlsh_set_tuning(h, C.byref(t)), "detlsh_set_tuning")


def detlsh_autotune(h, queries, k, beta=0.1, c=1.5, precision=PREC_FP32, rerank_mult=0,
                    cache_path=None, stream=None):
    """Choose the query kernel's knobs on a sample of queries; returns
    (Tuning, from_cache)."""
    qp = detlsh_default_query_params()
    qp.beta, qp.c, qp.precision, qp.rerank_mult = beta, c, precision, rerank_mult
    t, fc = Tuning(), C.c_int32(0)
    path = os.fsencode(cache_path) if cache_path is not None else None
    _check(lib().detlsh_autotune(h, _ptr(queries), queries.shape[0], k, C.byref(qp), path,
                                 _stream_ptr(stream), C.byref(t), C.byref(fc)), "detlsh_autotune")
    return t, bool(fc.value)


def detlsh_free(h):
    if h:
        lib().detlsh_free(h)


def detlsh_query_ex(h, queries, k, beta=0.1, c=1.5, precision=PREC_FP32, rerank_mult=0,
                    k_per_query=None, stream=None, ids=None, dists=None, r_min=None,
                    rmin_policy=None, per_tree=False):
    """Returns (ids int64 (m, k), dists float32 (m, k)); torch CUDA if queries are.
    r_min given: Alg. 5 from that radius with condition 2 (RMIN_FIXED);
    rmin_policy=RMIN_CONTINUOUS: the smallest r_min off the grid."""
    m = queries.shape[0]
    qp = detlsh_default_query_params()
    qp.beta, qp.c, qp.precision, qp.rerank_mult = beta, c, precision, rerank_mult
    if r_min is not None:
        qp.rmin_policy, qp.r_min = RMIN_FIXED, r_min
    if rmin_policy is not None:
        qp.rmin_policy = rmin_policy
    qp.per_tree = int(per_tree)
    if ids is None:
        if _is_cuda(queries):
            import torch
            ids = torch.empty((m, k), dtype=torch.int64, device=queries.device)
            dists = torch.empty((m, k), dtype=torch.float32, device=queries.device)
        else:
            ids = np.empty((m, k), np.int64)
            dists = np.empty((m, k), np.float32)
    kq = None
    if k_per_query is not None:
        kq = np.ascontiguousarray(k_per_query, np.int32)
    _check(lib().detlsh_query_ex(h, _ptr(queries), m, _ptr(kq), k, C.byref(qp),
                                 _stream_ptr(stream), _ptr(ids), _ptr(dists)), "detlsh_query_ex")
    return ids, dists


def detlsh_query_noalloc(h, queries, k, beta=0.1, c=1.5, precision=PREC_FP32, rerank_mult=0,
                         stream=None, ids=None, dists=None, per_tree=False):
    """Queries answered with the library's fixed scratch array: the call
    allocates no device memory (for callers that cannot allocate while
    serving).  queries, ids and dists must be CUDA tensors; ids/dists are
    allocated here by torch when not given."""
    import torch
    m = queries.shape[0]
    qp = detlsh_default_query_params()
    qp.beta, qp.c, qp.precision, qp.rerank_mult = beta, c, precision, rerank_mult
    qp.per_tree = int(per_tree)
    if ids is None:
        ids = torch.empty((m, k), dtype=torch.int64, device=queries.device)
        dists = torch.empty((m, k), dtype=torch.float32, device=queries.device)
    _check(lib().detlsh_query_noalloc(h, _ptr(queries), m, k, C.byref(qp), _stream_ptr(stream),
                                      _ptr(ids), _ptr(dists)), "detlsh_query_noalloc")
    return ids, dists


def detlsh_query(h, queries, k, c=1.5):
    m = queries.shape[0]
    ids = np.empty((m, k), np.int64)
    dists = np.empty((m, k), np.float32)
    _check(lib().detlsh_query(h, _ptr(queries), m, k, c, _ptr(ids), _ptr(dists)), "detlsh_query")
    return ids, dists


def detlsh_get_info(h):
    info = Info()
    _check(lib().detlsh_get_info(h, C.byref(info)), "detlsh_get_info")
    return info


def detlsh_get_projection_matrix(h):
    i = detlsh_get_info(h)
    A = np.empty((i.L * i.K, i.d), np.float32)
    _check(lib().detlsh_get_projection_matrix(h, _ptr(A)), "detlsh_get_projection_matrix")
    return A


def detlsh_get_sample(h):
    i = detlsh_get_info(h)
    s = np.empty(max(i.sample_size, 1), np.int64)
    _check(lib().detlsh_get_sample(h, _ptr(s)), "detlsh_get_sample")
    return s[:i.sample_size]


def detlsh_get_breakpoints(h):
    i = detlsh_get_info(h)
    B = np.empty((i.L * i.K, i.N_r + 1), np.float32)
    _check(lib().detlsh_get_breakpoints(h, _ptr(B)), "detlsh_get_breakpoints")
    return B


def detlsh_get_codes(h):
    i = detlsh_get_info(h)
    c = np.empty((i.n, i.L * i.K), np.uint8)
    _check(lib().detlsh_get_codes(h, _ptr(c)), "detlsh_get_codes")
    return c


def detlsh_get_projections(h):
    i = detlsh_get_info(h)
    P = np.empty((i.n, i.L * i.K), np.float32)
    _check(lib().detlsh_get_projections(h, _ptr(P)), "detlsh_get_projections")
    return P


def detlsh_get_tree(h, t):
    i = detlsh_get_info(h)
    nl = i.num_leaves[t]
    out = dict(perm=np.empty(i.n, np.int64), begin=np.empty(nl + 1, np.int64),
               lo=np.empty((nl, i.K), np.uint8), hi=np.empty((nl, i.K), np.uint8),
               nb=np.empty((nl, i.K), np.uint8), leaf_of=np.empty(i.n, np.int64))
    _check(lib().detlsh_get_tree(h, t, _ptr(out["perm"]), _ptr(out["begin"]), _ptr(out["lo"]),
                                 _ptr(out["hi"]), _ptr(out["nb"]), _ptr(out["leaf_of"])),
           "detlsh_get_tree")
    return out


def detlsh_get_timings(h):
    t = Timings()
    _check(lib().detlsh_get_timings(h, C.byref(t)), "detlsh_get_timings")
    return t


def detlsh_get_level_table(h, c):
    T = np.empty(255, np.float32)
    _check(lib().detlsh_get_level_table(h, c, _ptr(T)), "detlsh_get_level_table")
    return T


def detlsh_project(h, rows, stream=None):
    i = detlsh_get_info(h)
    m = rows.shape[0]
    if _is_cuda(rows):
        import torch
        out = torch.empty((m, i.L * i.K), dtype=torch.float32, device=rows.device)
    else:
        out = np.empty((m, i.L * i.K), np.float32)
    _check(lib().detlsh_project(h, _ptr(rows), m, _ptr(out), _stream_ptr(stream)),
           "detlsh_project")
    return out


def detlsh_query_candidates(h, queries, k, beta=0.1, c=1.5, cap=None, r_min=None,
                            rmin_policy=None, per_tree=False):
    """Candidate sets of Alg. 5: list of id arrays, j*, i* per query (with r_min:
    the stopping radius index and tree, -1 for condition 2)."""
    i = detlsh_get_info(h)
    m = queries.shape[0]
    cap = i.n if cap is None else cap
    qp = detlsh_default_query_params()
    qp.beta, qp.c = beta, c
    if r_min is not None:
        qp.rmin_policy, qp.r_min = RMIN_FIXED, r_min
    if rmin_policy is not None:
        qp.rmin_policy = rmin_policy
    qp.per_tree = int(per_tree)
    S = np.empty((m, cap), np.int64)
    ssz = np.empty(m, np.int64)
    js = np.empty(m, np.int32)
    ist = np.empty(m, np.int32)
    _check(lib().detlsh_query_candidates(h, _ptr(queries), m, k, C.byref(qp), cap, _ptr(S),
                                         _ptr(ssz), _ptr(js), _ptr(ist)),
           "detlsh_query_candidates")
    return [S[r, :ssz[r]].copy() for r in range(m)], js, ist


def detlsh_query_reserve(h, m_max, k_max, beta=0.1, c=1.5, precision=PREC_FP32, rerank_mult=0,
                         r_min=None):
    """Fix the parameters and sizes of detlsh_query_async and allocate its buffers."""
    qp = detlsh_default_query_params()
    qp.beta, qp.c, qp.precision, qp.rerank_mult = beta, c, precision, rerank_mult
    if r_min is not None:
        qp.rmin_policy, qp.r_min = RMIN_FIXED, r_min
    _check(lib().detlsh_query_reserve(h, m_max, k_max, C.byref(qp)), "detlsh_query_reserve")


def detlsh_query_async(h, queries, k_max, ids, dists, status, k_per_query=None, stream=None):
    """Enqueue one batch (device tensors only); capturable in a CUDA graph.
    Device-side errors land in status (int32 tensor of one element)."""
    _check(lib().detlsh_query_async(h, _ptr(queries), queries.shape[0], _ptr(k_per_query), k_max,
                                    _stream_ptr(stream), _ptr(ids), _ptr(dists), _ptr(status)),
           "detlsh_query_async")


def detlsh_rc_ann(h, queries, r, beta=0.1, c=1.5, S_cap=0, stream=None, optimised=False):
    """Alg. 4 (r,c)-ANN: ids (-1 = nothing), dists, tree_stop, S_size, and S
    (list of id arrays) when S_cap > 0.  Host numpy or CUDA tensors in; numpy out."""
    m = queries.shape[0]
    ids = np.empty(m, np.int64)
    dists = np.empty(m, np.float32)
    stop = np.empty(m, np.int32)
    ssz = np.empty(m, np.int64)
    S = np.empty((m, S_cap), np.int64) if S_cap > 0 else None
    _check(lib().detlsh_rc_ann(h, _ptr(queries), m, r, beta, c, int(optimised),
                               _stream_ptr(stream), _ptr(ids),
                               _ptr(dists), _ptr(stop), S_cap, _ptr(S) if S is not None else None,
                               _ptr(ssz)),
           "detlsh_rc_ann")
    Sl = [S[i, :min(ssz[i], S_cap)].copy() for i in range(m)] if S is not None else None
    return ids, dists, stop, ssz, Sl


class Index:
    """Owning wrapper: builds on construction, frees on close/garbage collection."""

    def __init__(self, data, **kw):
        self.h = detlsh_build(data, **kw)

    def close(self):
        if getattr(self, "h", None):
            detlsh_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def query(self, queries, k, **kw):
        return detlsh_query_ex(self.h, queries, k, **kw)

    def info(self):
        return detlsh_get_info(self.h)
