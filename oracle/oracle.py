"""ctypes wrapper of liboracle.so: numpy in, numpy out.  Test infrastructure only."""
import ctypes as C
import os

import numpy as np

from .build import build_oracle

_lib = None
NLEV = 255
JMIN = -127

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")


def _nullable(base):
    """ndpointer type that also accepts None (passed as NULL)."""
    def from_param(cls, obj):
        if obj is None:
            return None
        return base.from_param(obj)
    return type(base.__name__ + "_or_null", (base,), {"from_param": classmethod(from_param)})


_i64p_n = _nullable(_i64p)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_projection_matrix.argtypes = [C.c_int, C.c_int64, C.c_uint64, _f32p]
        L.orc_dot_rn32.argtypes = [_f32p, _f32p, C.c_int64]
        L.orc_dot_rn32.restype = C.c_float
        L.orc_dist2_le.argtypes = [_f32p, _f32p, C.c_int64, C.c_double]
        L.orc_dist2_le.restype = C.c_int
        L.orc_project.argtypes = [_f32p, C.c_int64, C.c_int64, _f32p, C.c_int, _f32p]
        L.orc_sample.argtypes = [C.c_int64, C.c_uint64, C.c_double, C.c_int, _i64p]
        L.orc_sample.restype = C.c_int64
        L.orc_breakpoints.argtypes = [_f32p, C.c_int64, C.c_int, _i64p, C.c_int64, C.c_int, _f32p]
        L.orc_encode.argtypes = [_f32p, C.c_int64, C.c_int, _f32p, C.c_int, _u8p]
        L.orc_chi2_sf.argtypes = [C.c_double, C.c_int]
        L.orc_chi2_sf.restype = C.c_double
        L.orc_eps2.argtypes = [C.c_int, C.c_int]
        L.orc_eps2.restype = C.c_double
        L.orc_level_table.argtypes = [C.c_double, C.c_double, _f32p]
        L.orc_index_build.argtypes = [_f32p, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int,
                                      C.c_uint64, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_static_breakpoints.argtypes = [C.c_int, C.c_int, _f32p]
        L.orc_index_build.restype = C.c_void_p
        L.orc_index_free.argtypes = [C.c_void_p]
        L.orc_index_sample_size.argtypes = [C.c_void_p]
        L.orc_index_sample_size.restype = C.c_int64
        L.orc_index_num_leaves.argtypes = [C.c_void_p, C.c_int]
        L.orc_index_num_leaves.restype = C.c_int64
        L.orc_index_export_arrays.argtypes = [C.c_void_p, _f32p, _f32p, _u8p, _f32p, _i64p]
        L.orc_index_export_tree.argtypes = [C.c_void_p, C.c_int, _i64p, _i64p, _u8p, _u8p,
                                            _u8p, _i64p]
        L.orc_index_level_table.argtypes = [C.c_void_p, C.c_double, _f32p]
        L.orc_index_query.argtypes = [C.c_void_p, _f32p, C.c_int, C.c_double, C.c_double,
                                      _i64p, _f64p, _i64p_n, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_index_query.restype = C.c_int
        L.orc_index_query_ex.argtypes = [C.c_void_p, _f32p, C.c_int, C.c_double, C.c_double,
                                         C.c_int, _i64p, _f64p, _i64p_n, C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_index_query_ex.restype = C.c_int
        L.orc_index_query_fixed.argtypes = [C.c_void_p, _f32p, C.c_int, C.c_double, C.c_double,
                                            C.c_double, _i64p, _f64p, _i64p_n,
                                            C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                            C.POINTER(C.c_int)]
        L.orc_index_query_fixed.restype = C.c_int
        L.orc_index_query_magic_min.argtypes = [C.c_void_p, _f32p, C.c_int, C.c_double, _i64p,
                                                _f64p, _i64p_n, C.POINTER(C.c_int64),
                                                C.POINTER(C.c_float), C.POINTER(C.c_int)]
        L.orc_index_query_magic_min.restype = C.c_int
        L.orc_index_query_batch.argtypes = [C.c_void_p, _f32p, C.c_int64, C.c_int, C.c_double,
                                            C.c_double, _i64p, _f64p, _i64p, C.c_int]
        L.orc_index_query_batch.restype = C.c_int
        L.orc_index_leaf_lb2.argtypes = [C.c_void_p, C.c_int, _f32p, _f32p]
        L.orc_index_leaf_ub2.argtypes = [C.c_void_p, C.c_int, _f32p, _f32p]
        L.orc_box_bounds.argtypes = [_f32p, C.c_int, C.c_int, _f32p, _u8p, _u8p,
                                     C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.orc_index_range_exact.argtypes = [C.c_void_p, C.c_int, _f32p, C.c_double, _i64p]
        L.orc_index_range_exact.restype = C.c_int64
        L.orc_index_rc_ann.argtypes = [C.c_void_p, _f32p, C.c_double, C.c_double, C.c_double,
                                       C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double), _i64p_n,
                                       C.POINTER(C.c_int64), C.POINTER(C.c_int)]
        L.orc_index_rc_ann.restype = C.c_int
        L.orc_bruteforce_knn.argtypes = [_f32p, C.c_int64, C.c_int64, _f32p, C.c_int64, C.c_int,
                                         _i64p, _f64p, C.c_int]
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def box_bounds(B, q, lo, hi):
    """(LB^2, UB^2) of the box [B[j][lo_j], B[j][hi_j + 1]] to q (Sec. IV-C)."""
    B = _f32(B)
    K, R = B.shape
    lb, ub = C.c_float(), C.c_float()
    lib().orc_box_bounds(B, K, R - 1, _f32(q), np.ascontiguousarray(lo, np.uint8),
                         np.ascontiguousarray(hi, np.uint8), C.byref(lb), C.byref(ub))
    return lb.value, ub.value


def projection_matrix(LK, d, seed):
    A = np.zeros((LK, d), np.float32)
    lib().orc_projection_matrix(LK, d, seed, A)
    return A


def dot_rn32(a, x):
    a, x = _f32(a), _f32(x)
    return np.float32(lib().orc_dot_rn32(a, x, a.size))


def dist_le(q, x, R):
    """Exact ||q - x|| <= R (condition 2 of Alg. 5): 1 within, 0 beyond, -1 out of range."""
    q, x = _f32(q), _f32(x)
    return int(lib().orc_dist2_le(q, x, q.size, float(R)))


def project(X, A):
    X, A = _f32(X), _f32(A)
    n, d = X.shape
    P = np.zeros((n, A.shape[0]), np.float32)
    lib().orc_project(X, n, d, A, A.shape[0], P)
    return P


def sample(n, seed, frac, N_r):
    ids = np.zeros(max(n, 1), np.int64)
    m = lib().orc_sample(n, seed, frac, N_r, ids)
    return ids[:m].copy()


def breakpoints(P, sample_ids, N_r):
    P = _f32(P)
    n, LK = P.shape
    s = np.ascontiguousarray(sample_ids, np.int64)
    B = np.zeros((LK, N_r + 1), np.float32)
    lib().orc_breakpoints(P, n, LK, s, s.size, N_r, B)
    return B


def static_breakpoints(LK, N_r):
    """Static encoding scheme (Sec. III-A): N(0,1) equal-mass breakpoints."""
    B = np.zeros((LK, N_r + 1), np.float32)
    lib().orc_static_breakpoints(LK, N_r, B)
    return B


def encode(P, B):
    P, B = _f32(P), _f32(B)
    n, LK = P.shape
    codes = np.zeros((n, LK), np.uint8)
    lib().orc_encode(P, n, LK, B, B.shape[1] - 1, codes)
    return codes


def chi2_sf(x, K):
    return lib().orc_chi2_sf(x, K)


def eps2(K, L):
    return lib().orc_eps2(K, L)


def level_table(e2, c):
    T = np.zeros(NLEV, np.float32)
    lib().orc_level_table(e2, c, T)
    return T


class Index:
    """Oracle index: encoding (Alg. 1) + L pointer-based DE-Trees (Alg. 2)."""

    def __init__(self, X, L=4, K=16, N_r=256, seed=0, frac=0.1, M=64, box_mode=0,
                 insertion_order=0, encoding=0):
        X = _f32(X)
        self.n, self.d = X.shape
        self.L, self.K, self.N_r, self.M = L, K, N_r, M
        self.X = X
        self._h = lib().orc_index_build(X, self.n, self.d, L, K, N_r, seed, frac, M,
                                        box_mode, insertion_order, encoding)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_index_free(self._h)
            self._h = None

    def arrays(self):
        LK = self.L * self.K
        m = lib().orc_index_sample_size(self._h)
        A = np.zeros((LK, self.d), np.float32)
        B = np.zeros((LK, self.N_r + 1), np.float32)
        codes = np.zeros((self.n, LK), np.uint8)
        P = np.zeros((self.n, LK), np.float32)
        s = np.zeros(max(m, 1), np.int64)
        lib().orc_index_export_arrays(self._h, A, B, codes, P, s)
        return dict(A=A, B=B, codes=codes, P=P, sample=s[:m])

    def num_leaves(self, t):
        return lib().orc_index_num_leaves(self._h, t)

    def tree(self, t):
        nl = self.num_leaves(t)
        perm = np.zeros(self.n, np.int64)
        begin = np.zeros(nl + 1, np.int64)
        lo = np.zeros((nl, self.K), np.uint8)
        hi = np.zeros((nl, self.K), np.uint8)
        nb = np.zeros((nl, self.K), np.uint8)
        leaf_of = np.zeros(self.n, np.int64)
        lib().orc_index_export_tree(self._h, t, perm, begin, lo, hi, nb, leaf_of)
        return dict(perm=perm, begin=begin, lo=lo, hi=hi, nb=nb, leaf_of=leaf_of)

    def level_table(self, c):
        T = np.zeros(NLEV, np.float32)
        lib().orc_index_level_table(self._h, c, T)
        return T

    def leaf_lb2(self, t, q):
        out = np.zeros(self.num_leaves(t), np.float32)
        lib().orc_index_leaf_lb2(self._h, t, _f32(q), out)
        return out

    def leaf_ub2(self, t, q):
        out = np.zeros(self.num_leaves(t), np.float32)
        lib().orc_index_leaf_ub2(self._h, t, _f32(q), out)
        return out

    def range_exact(self, t, q, r):
        """Alg. 3 without the Sec. VI-B2 optimisations: ids within eps*r in tree t."""
        out = np.zeros(max(self.n, 1), np.int64)
        cnt = lib().orc_index_range_exact(self._h, t, _f32(q), r, out)
        return out[:cnt]

    def rc_ann(self, q, r, beta=0.1, c=1.5, want_S=True, optimised=False):
        """Alg. 4: (r,c)-ANN.  id -1 when the query returns nothing.  optimised:
        whole leaves by lower bound (Sec. VI-B2 (1)) instead of Alg. 3 as printed."""
        pid, dist = C.c_int64(0), C.c_double(0.0)
        ssz, stop = C.c_int64(0), C.c_int(0)
        S = np.zeros(max(self.n, 1), np.int64) if want_S else None
        lib().orc_index_rc_ann(self._h, _f32(q), r, beta, c, int(optimised), C.byref(pid),
                               C.byref(dist), S,
                               C.byref(ssz), C.byref(stop))
        return dict(id=pid.value, dist=dist.value, S=S[:ssz.value] if want_S else None,
                    S_size=ssz.value, tree_stop=stop.value)

    def query(self, q, k, beta=0.1, c=1.5, want_S=True, per_tree=False):
        ids = np.zeros(k, np.int64)
        dists = np.zeros(k, np.float64)
        S = np.zeros(self.n, np.int64) if want_S else np.zeros(1, np.int64)
        ssz, js, ist = C.c_int64(0), C.c_int(0), C.c_int(0)
        rc = lib().orc_index_query_ex(self._h, _f32(q), k, beta, c, int(per_tree), ids, dists,
                                      S if want_S else None, C.byref(ssz), C.byref(js),
                                      C.byref(ist))
        if rc != 0:
            raise ValueError("oracle query rejected its arguments")
        return dict(ids=ids, dists=dists, S=S[:ssz.value] if want_S else None,
                    S_size=ssz.value, jstar=js.value, istar=ist.value)

    def query_fixed(self, q, k, r_min, beta=0.1, c=1.5, want_S=True):
        """Alg. 5 from a fixed r_min with condition 2 (jstop: radius index,
        istop: tree for condition 1, -1 for condition 2)."""
        ids = np.zeros(k, np.int64)
        dists = np.zeros(k, np.float64)
        S = np.zeros(max(self.n, 1), np.int64) if want_S else None
        ssz, js, ist = C.c_int64(0), C.c_int(0), C.c_int(0)
        rc = lib().orc_index_query_fixed(self._h, _f32(q), k, beta, c, r_min, ids, dists, S,
                                         C.byref(ssz), C.byref(js), C.byref(ist))
        if rc != 0:
            raise ValueError("oracle query rejected its arguments")
        return dict(ids=ids, dists=dists, S=S[:ssz.value] if want_S else None,
                    S_size=ssz.value, jstop=js.value, istop=ist.value)

    def query_magic_min(self, q, k, beta=0.1, want_S=True):
        """Alg. 5 at the smallest continuous r_min (vstar: the squared threshold)."""
        ids = np.zeros(k, np.int64)
        dists = np.zeros(k, np.float64)
        S = np.zeros(max(self.n, 1), np.int64) if want_S else None
        ssz, vs, ist = C.c_int64(0), C.c_float(0.0), C.c_int(0)
        rc = lib().orc_index_query_magic_min(self._h, _f32(q), k, beta, ids, dists, S,
                                             C.byref(ssz), C.byref(vs), C.byref(ist))
        if rc != 0:
            raise ValueError("oracle query rejected its arguments")
        return dict(ids=ids, dists=dists, S=S[:ssz.value] if want_S else None,
                    S_size=ssz.value, vstar=vs.value, istar=ist.value)

    def query_batch(self, Q, k, beta=0.1, c=1.5, nthreads=0):
        Q = _f32(Q)
        m = Q.shape[0]
        ids = np.zeros((m, k), np.int64)
        dists = np.zeros((m, k), np.float64)
        ssz = np.zeros(m, np.int64)
        rc = lib().orc_index_query_batch(self._h, Q, m, k, beta, c, ids, dists, ssz, nthreads)
        if rc != 0:
            raise ValueError("oracle query rejected its arguments")
        return ids, dists, ssz


def bruteforce_knn(X, Q, k, nthreads=0):
    X, Q = _f32(X), _f32(Q)
    n, d = X.shape
    m = Q.shape[0]
    ids = np.zeros((m, k), np.int64)
    dists = np.zeros((m, k), np.float64)
    lib().orc_bruteforce_knn(X, n, d, Q, m, k, ids, dists, nthreads)
    return ids, dists
