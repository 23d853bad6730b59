"""Python binding of libmrf (include/mrf.h): argument marshalling only.

Every function of the C ABI is exposed under its own name (mrf_create,
mrf_set_factors, mrf_sweep, ...) through ctypes; the class `MRF` wraps a
handle.  Arrays may be numpy arrays (host memory) or torch tensors (host or
CUDA memory); PyTorch supplies device memory and the CUDA stream.  All
sampling runs in the library's CUDA kernels.  There is no fallback: if
libmrf.so has not been built, loading raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrf.so")

MRF_OK, MRF_EINVAL, MRF_ENONFINITE, MRF_ENOMEM, MRF_ECUDA, MRF_ERANGE, MRF_ETIMEOUT, MRF_ESTATE = range(8)
MRF_PTR_HOST, MRF_PTR_DEVICE = 0, 1
MODE_PLAIN, MODE_FUSED, MODE_SPLASH, MODE_LEARNED, MODE_SW, MODE_HIGDON = 0, 1, 2, 3, 4, 5
# status bits of a queue round's edit (mrf.h MRF_Q_*)
Q_COUNT, Q_GRAPH, Q_VERTEX, Q_LOOP, Q_SLOT, Q_DUP, Q_NONFINITE, Q_OFFDIAG, Q_PAIR, Q_SLOTS, Q_UNSORTED = \
    1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024
LAYOUT_PIVOT, LAYOUT_DIAG = 0, 1
(K_DUAL, K_PRIMAL, K_FUSED, K_POTENTIAL, K_FFBS, K_ACCUMULATE, K_FEATURES, K_MLP, K_MH, K_SMALL,
 K_SW_BOND, K_SW_FLATTEN, K_SW_DRAW, K_SW_SMALL, K_PARTIAL, K_COUNT) = range(16)
KERNEL_NAMES = ["k_dual", "k_primal", "k_primal<fused>", "k_potential", "k_ffbs", "k_accumulate",
                "k_learned_features", "k_mlp", "k_learned_mh", "k_sweep_small",
                "k_sw_bond", "k_sw_flatten", "k_sw_draw", "k_sw_small", "k_edge_partial"]


class mrf_options(ct.Structure):
    _fields_ = [("grid_nx", ct.c_int32), ("grid_ny", ct.c_int32), ("grid_nz", ct.c_int32),
                ("record_logp", ct.c_int32), ("use_graphs", ct.c_int32), ("schedule", ct.c_int32),
                ("kernel_timing", ct.c_int32), ("exact_edges", ct.c_int32), ("mlp_path", ct.c_int32),
                ("reserved", ct.c_int32 * 5)]


class mrf_info(ct.Structure):
    _fields_ = [("n_vars", ct.c_int32), ("n_labels", ct.c_int32), ("n_chains", ct.c_int32),
                ("layout", ct.c_int32), ("n_entries", ct.c_int32), ("n_edges", ct.c_int64),
                ("n_edge_slots", ct.c_int64), ("sweep_index", ct.c_int64), ("n_samples", ct.c_int64),
                ("log_const", ct.c_double), ("schedule", ct.c_int32), ("tune_ms_thread", ct.c_float),
                ("tune_ms_cta", ct.c_float)]


_P = ct.c_void_p
_SIGS = {
    "mrf_default_options": (None, [ct.POINTER(mrf_options)]),
    "mrf_create": (ct.c_int, [ct.POINTER(_P), ct.c_int32, ct.c_int32, ct.c_int32, ct.c_uint64,
                              ct.POINTER(mrf_options), _P]),
    "mrf_set_factors": (ct.c_int, [_P, _P, ct.c_int64, _P, _P, _P, ct.c_int32]),
    "mrf_edit_factors": (ct.c_int, [_P, ct.c_int64, _P, ct.c_int64, _P, _P, _P, _P, ct.c_int32]),
    "mrf_sweep": (ct.c_int, [_P, ct.c_int32, ct.c_int32]),
    "mrf_marginals": (ct.c_int, [_P, _P, ct.POINTER(ct.c_int64), ct.c_int32]),
    "mrf_get_counts": (ct.c_int, [_P, _P, ct.c_int32]),
    "mrf_reset_marginals": (ct.c_int, [_P, ct.c_int32]),
    "mrf_get_labels": (ct.c_int, [_P, _P, ct.c_int32]),
    "mrf_set_labels": (ct.c_int, [_P, _P, ct.c_int32]),
    "mrf_set_sweep_index": (ct.c_int, [_P, ct.c_int64]),
    "mrf_get_info": (ct.c_int, [_P, ct.POINTER(mrf_info)]),
    "mrf_debug_tables": (ct.c_int, [_P, _P, _P, _P]),
    "mrf_debug_logp": (ct.c_int, [_P, _P, ct.POINTER(ct.c_uint64)]),
    "mrf_debug_theta": (ct.c_int, [_P, _P]),
    "mrf_kernel_times": (ct.c_int, [_P, _P, _P]),
    "mrf_set_kernel_timing": (ct.c_int, [_P, ct.c_int32]),
    "mrf_estimate_log_partition": (ct.c_int, [_P, ct.c_int32, _P]),
    "mrf_estimate_log_partition_sw": (ct.c_int, [_P, ct.c_int32, _P]),
    "mrf_set_higdon": (ct.c_int, [_P, ct.c_double]),
    "mrf_estimate_log_partition_higdon": (ct.c_int, [_P, ct.c_int32, _P]),
    "mrf_map_em": (ct.c_int, [_P, ct.c_int32, _P, ct.c_int32]),
    "mrf_save": (ct.c_int, [_P, ct.c_char_p]),
    "mrf_load": (ct.c_int, [ct.POINTER(_P), ct.c_char_p, _P]),
    "mrf_map_em_blocked": (ct.c_int, [_P, ct.c_int32, _P, ct.c_int32]),
    "mrf_mean_field": (ct.c_int, [_P, ct.c_int32, _P, ct.c_int32]),
    "mrf_mean_field_blocked": (ct.c_int, [_P, ct.c_int32, _P, ct.c_int32]),
    "mrf_philox_rate": (ct.c_int, [ct.c_uint64, ct.c_int32, _P, ct.POINTER(ct.c_double)]),
    "mrf_sweep_noalloc": (ct.c_int, [_P, _P, _P, ct.c_int64]),
    "mrf_learned_setup": (ct.c_int, [_P, _P, ct.c_int32, ct.c_uint64]),
    "mrf_learned_param_count": (ct.c_int64, [_P]),
    "mrf_learned_set_params": (ct.c_int, [_P, _P, ct.c_int64]),
    "mrf_learned_get_params": (ct.c_int, [_P, _P, ct.c_int64]),
    "mrf_learned_harvest": (ct.c_int, [_P, ct.c_int32, ct.c_int32, ct.c_int64, ct.POINTER(ct.c_int64)]),
    "mrf_learned_train": (ct.c_int, [_P, ct.c_int32, ct.c_int32, ct.c_float, ct.c_uint64, _P]),
    "mrf_learned_grad": (ct.c_int, [_P, _P, _P, _P, ct.c_int32, _P, ct.POINTER(ct.c_double)]),
    "mrf_learned_forward": (ct.c_int, [_P, _P, ct.c_int32, _P]),
    "mrf_learned_stats": (ct.c_int, [_P, ct.POINTER(ct.c_uint64), ct.POINTER(ct.c_uint64)]),
    "mrf_learned_debug": (ct.c_int, [_P, _P, _P]),
    "mrf_debug_mlp_timeout": (ct.c_int, [_P, ct.c_int32]),
    "mrf_batch_create": (ct.c_int, [ct.POINTER(_P), ct.c_int32, _P, _P, ct.c_int32, ct.c_uint64,
                                    ct.POINTER(mrf_options), _P]),
    "mrf_batch_set_factors": (ct.c_int, [_P, _P, _P, _P, _P, _P]),
    "mrf_batch_edit_factors": (ct.c_int, [_P, ct.c_int64, _P, _P, ct.c_int64, _P, _P, _P, _P, _P]),
    "mrf_batch_sweep": (ct.c_int, [_P, ct.c_int32, ct.c_int32]),
    "mrf_batch_queue_create": (ct.c_int, [_P, ct.c_int64, ct.c_int64, ct.c_int64, ct.c_int64]),
    "mrf_batch_queue_load": (ct.c_int, [_P, ct.c_int64, _P, _P, ct.c_int64, _P, _P, _P, ct.c_int64, _P, ct.c_int32]),
    "mrf_batch_round": (ct.c_int, [_P, ct.c_int32, ct.c_int32]),
    "mrf_batch_set_kernel_timing": (ct.c_int, [_P, ct.c_int32]),
    "mrf_batch_queue_result": (ct.c_int, [_P, ct.POINTER(ct.c_uint32), ct.c_int64, _P]),
    "mrf_batch_reset_marginals": (ct.c_int, [_P, ct.c_int32]),
    "mrf_batch_get_counts": (ct.c_int, [_P, ct.c_int32, _P]),
    "mrf_batch_get_labels": (ct.c_int, [_P, ct.c_int32, _P]),
    "mrf_batch_graph": (ct.c_int, [_P, ct.c_int32, _P]),
    "mrf_batch_n_classes": (ct.c_int32, [_P]),
    "mrf_batch_class": (_P, [_P, ct.c_int32]),
    "mrf_batch_last_error": (ct.c_char_p, [_P]),
    "mrf_batch_destroy": (None, [_P]),
    "mrf_last_error": (ct.c_char_p, [_P]),
    "mrf_status_string": (ct.c_char_p, [ct.c_int]),
    "mrf_destroy": (None, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libmrf.so and declare every exported signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1611_06684_gb300.build.build()")
    lib = ct.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


class MrfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def _ptr(a):
    """(pointer, ptr_kind, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, MRF_PTR_HOST, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, MRF_PTR_HOST, a
    import torch  # noqa: F401  (only for tensors)
    t = a.contiguous()
    return t.data_ptr(), (MRF_PTR_DEVICE if t.is_cuda else MRF_PTR_HOST), t


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


class MRF:
    """Owner of one mrf_t handle (see include/mrf.h for semantics)."""

    def __init__(self, n_vars: int, n_labels: int, n_chains: int, seed: int = 0, grid=None,
                 record_logp: bool = False, use_graphs: bool = True, schedule: int = 0, stream=None,
                 kernel_timing: bool = False, exact_edges: bool = False, mlp_path: int = 0):
        lib = load()
        opt = mrf_options()
        lib.mrf_default_options(ct.byref(opt))
        if grid is not None:
            opt.grid_nx, opt.grid_ny, opt.grid_nz = (int(g) for g in grid)
        opt.record_logp = int(record_logp)
        opt.use_graphs = int(use_graphs)
        opt.schedule = int(schedule)
        opt.kernel_timing = int(kernel_timing)
        opt.exact_edges = int(exact_edges)
        opt.mlp_path = int(mlp_path)
        self.stream = _current_stream() if stream is None else int(stream)
        h = _P()
        st = lib.mrf_create(ct.byref(h), n_vars, n_labels, n_chains, ct.c_uint64(seed & (2**64 - 1)), ct.byref(opt),
                            _P(self.stream))
        if st != MRF_OK:
            raise MrfError(st, lib.mrf_status_string(st).decode())
        self.h = h
        self.lib = lib
        self.N, self.L, self.C = n_vars, n_labels, n_chains

    def _check(self, st):
        if st != MRF_OK:
            raise MrfError(st, self.lib.mrf_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) and not getattr(self, "_borrowed", False):
            self.lib.mrf_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- model
    def set_factors(self, unary, src, dst, pair):
        pu, ku, a = _ptr(unary); ps, ks, b = _ptr(src); pd, kd, c = _ptr(dst); pp, kp, d = _ptr(pair)
        kinds = {ku, ks, kd, kp} if int(np.prod(np.shape(src))) else {ku}
        if len(kinds) != 1:
            raise ValueError("all arrays must be on the same side (host or device)")
        n = int(np.prod(src.shape)) if src is not None else 0
        self._check(self.lib.mrf_set_factors(self.h, pu, n, ps, pd, pp, ku))

    def edit_factors(self, remove_ids, src, dst, pair):
        rem = np.ascontiguousarray(remove_ids, np.int64)
        s = np.ascontiguousarray(src, np.int32); t = np.ascontiguousarray(dst, np.int32)
        p = np.ascontiguousarray(pair, np.float32)
        out = np.zeros(s.shape[0], np.int64)
        self._check(self.lib.mrf_edit_factors(self.h, rem.shape[0], rem.ctypes.data, s.shape[0], s.ctypes.data,
                                              t.ctypes.data, p.ctypes.data, out.ctypes.data, MRF_PTR_HOST))
        return out

    # -- sampling
    def sweep(self, n: int = 1, mode: int = MODE_PLAIN):
        self._check(self.lib.mrf_sweep(self.h, int(n), int(mode)))

    def set_higdon(self, rho: float):
        """Fraction rho of Higdon's partial Swendsen-Wang sweep (MODE_HIGDON)."""
        self._check(self.lib.mrf_set_higdon(self.h, float(rho)))

    def reset_marginals(self, burn_in: int = 0):
        self._check(self.lib.mrf_reset_marginals(self.h, int(burn_in)))

    def marginals(self):
        out = np.zeros((self.N, self.L), np.float32)
        ns = ct.c_int64()
        self._check(self.lib.mrf_marginals(self.h, out.ctypes.data, ct.byref(ns), MRF_PTR_HOST))
        return out, ns.value

    def counts(self):
        out = np.zeros((self.N, self.L), np.uint32)
        self._check(self.lib.mrf_get_counts(self.h, out.ctypes.data, MRF_PTR_HOST))
        return out

    def get_labels(self):
        out = np.zeros((self.C, self.N), np.uint8)
        self._check(self.lib.mrf_get_labels(self.h, out.ctypes.data, MRF_PTR_HOST))
        return out

    def set_labels(self, x):
        p, k, keep = _ptr(np.ascontiguousarray(x, np.uint8) if isinstance(x, np.ndarray) else x)
        self._check(self.lib.mrf_set_labels(self.h, p, k))

    def get_labels_into(self, out):
        """Labels [C][N] into a caller buffer (numpy, pinned or CUDA torch tensor)."""
        p, k, keep = _ptr(out)
        self._check(self.lib.mrf_get_labels(self.h, p, k))
        return out

    def set_sweep_index(self, t: int):
        self._check(self.lib.mrf_set_sweep_index(self.h, int(t)))

    def info(self) -> mrf_info:
        inf = mrf_info()
        self._check(self.lib.mrf_get_info(self.h, ct.byref(inf)))
        return inf

    # -- debug / parity views
    def debug_tables(self):
        inf = self.info()
        tau = np.zeros((inf.n_edge_slots, inf.n_entries), np.float32)
        thr = np.zeros((inf.n_edge_slots, inf.n_entries), np.uint32)
        ut = np.zeros((self.N, self.L), np.float64)
        self._check(self.lib.mrf_debug_tables(self.h, tau.ctypes.data, thr.ctypes.data, ut.ctypes.data))
        return tau, thr, ut

    def debug_logp(self):
        out = np.zeros((self.C, self.N, self.L), np.float32)
        b = ct.c_uint64()
        self._check(self.lib.mrf_debug_logp(self.h, out.ctypes.data, ct.byref(b)))
        return out, b.value

    def boundary_draws(self) -> int:
        b = ct.c_uint64()
        self._check(self.lib.mrf_debug_logp(self.h, None, ct.byref(b)))
        return b.value

    def sweep_noalloc(self, labels_in, labels_out, sweep_index: int):
        """One plain sweep without device allocation (mrf_sweep_noalloc): labels
        are CUDA tensors [n_vars][n_chains] uint8 owned by the caller."""
        self._check(self.lib.mrf_sweep_noalloc(self.h, labels_in.data_ptr(), labels_out.data_ptr(), int(sweep_index)))

    # -- learned block proposal
    def learned_setup(self, block_of_site, hidden: int = 256, seed: int = 0):
        bos = np.ascontiguousarray(block_of_site, np.int32)
        self._check(self.lib.mrf_learned_setup(self.h, bos.ctypes.data, int(hidden), ct.c_uint64(seed)))
        self.n_params = int(self.lib.mrf_learned_param_count(self.h))

    def learned_set_params(self, flat):
        f = np.ascontiguousarray(flat, np.float32)
        self._check(self.lib.mrf_learned_set_params(self.h, f.ctypes.data, f.shape[0]))

    def learned_get_params(self):
        out = np.zeros(self.n_params, np.float32)
        self._check(self.lib.mrf_learned_get_params(self.h, out.ctypes.data, out.shape[0]))
        return out

    def learned_harvest(self, n_sweeps: int, stride: int, max_rows: int) -> int:
        rows = ct.c_int64()
        self._check(self.lib.mrf_learned_harvest(self.h, int(n_sweeps), int(stride), int(max_rows), ct.byref(rows)))
        return rows.value

    def learned_train(self, steps: int, batch: int, lr: float, seed: int = 0):
        trace = np.zeros(max(steps, 1), np.float32)
        self._check(self.lib.mrf_learned_train(self.h, int(steps), int(batch), ct.c_float(lr), ct.c_uint64(seed),
                                               trace.ctypes.data))
        return trace[:steps]

    def learned_grad(self, X, y, nmem):
        X = np.ascontiguousarray(X, np.float32); y = np.ascontiguousarray(y, np.uint8)
        n = np.ascontiguousarray(nmem, np.uint8)
        g = np.zeros(self.n_params, np.float32)
        loss = ct.c_double()
        self._check(self.lib.mrf_learned_grad(self.h, X.ctypes.data, y.ctypes.data, n.ctypes.data, X.shape[0],
                                              g.ctypes.data, ct.byref(loss)))
        return loss.value, g

    def learned_forward(self, X, n_out: int):
        X = np.ascontiguousarray(X, np.float32)
        z = np.zeros((X.shape[0], n_out), np.float32)
        self._check(self.lib.mrf_learned_forward(self.h, X.ctypes.data, X.shape[0], z.ctypes.data))
        return z

    def learned_stats(self):
        p, a = ct.c_uint64(), ct.c_uint64()
        self._check(self.lib.mrf_learned_stats(self.h, ct.byref(p), ct.byref(a)))
        return p.value, a.value

    def learned_debug(self, rows: int, width: int, n_out: int):
        X = np.zeros((rows, width), np.float32); z = np.zeros((rows, n_out), np.float32)
        self._check(self.lib.mrf_learned_debug(self.h, X.ctypes.data, z.ctypes.data))
        return X, z

    def estimate_log_partition(self, n_sweeps: int, mode: int = MODE_PLAIN):
        """log V [n_sweeps][C] of Section 5.2's estimator over n plain (or, with
        mode=MODE_SW / MODE_HIGDON, Swendsen-Wang / Higdon) sweeps."""
        out = np.zeros((int(n_sweeps), self.C), np.float64)
        fns = {MODE_PLAIN: self.lib.mrf_estimate_log_partition, MODE_SW: self.lib.mrf_estimate_log_partition_sw,
               MODE_HIGDON: self.lib.mrf_estimate_log_partition_higdon}
        if mode not in fns:
            raise ValueError("the estimator runs plain, Swendsen-Wang or Higdon sweeps")
        fn = fns[mode]
        self._check(fn(self.h, int(n_sweeps), out.ctypes.data))
        return out

    def save(self, path: str):
        """Checkpoint of the model and the chains (mrf_save)."""
        self._check(self.lib.mrf_save(self.h, str(path).encode()))

    @classmethod
    def load(cls, path: str, stream=None):
        """A handle resumed from a checkpoint (mrf_load)."""
        lib = load()
        st_ptr = _current_stream() if stream is None else int(stream)
        h = _P()
        st = lib.mrf_load(ct.byref(h), str(path).encode(), _P(st_ptr))
        if st != MRF_OK:
            raise MrfError(st, lib.mrf_status_string(st).decode())
        obj = cls.__new__(cls)
        inf = mrf_info()
        lib.mrf_get_info(h, ct.byref(inf))
        obj.h, obj.lib, obj.stream = h, lib, st_ptr
        obj.N, obj.L, obj.C = inf.n_vars, inf.n_labels, inf.n_chains
        return obj

    def map_em(self, labels, n_iters: int):
        """Primal-dual EM from labels [C][N]; returns the labels after n_iters iterations."""
        x = np.ascontiguousarray(labels, np.uint8).copy()
        self._check(self.lib.mrf_map_em(self.h, int(n_iters), x.ctypes.data, MRF_PTR_HOST))
        return x

    def map_em_blocked(self, labels, n_iters: int):
        """Blocked EM (lattice handles) from labels [C][N]; returns the labels after n_iters iterations."""
        x = np.ascontiguousarray(labels, np.uint8).copy()
        self._check(self.lib.mrf_map_em_blocked(self.h, int(n_iters), x.ctypes.data, MRF_PTR_HOST))
        return x

    def mean_field(self, marginals, n_iters: int):
        """Primal-dual mean field from marginals [C][N][L]; returns them after n_iters iterations."""
        q = np.ascontiguousarray(marginals, np.float32).copy()
        self._check(self.lib.mrf_mean_field(self.h, int(n_iters), q.ctypes.data, MRF_PTR_HOST))
        return q

    def mean_field_blocked(self, marginals, n_iters: int):
        """Tree (blocked) mean field from marginals [C][N][L] on a lattice handle."""
        q = np.ascontiguousarray(marginals, np.float32).copy()
        self._check(self.lib.mrf_mean_field_blocked(self.h, int(n_iters), q.ctypes.data, MRF_PTR_HOST))
        return q

    def debug_mlp_timeout(self, on: bool = True):
        """Arm the tensor-core MLP's timeout test hook for the next learned sweep."""
        self._check(self.lib.mrf_debug_mlp_timeout(self.h, int(bool(on))))

    def set_kernel_timing(self, on: bool):
        self._check(self.lib.mrf_set_kernel_timing(self.h, int(bool(on))))

    def kernel_times(self):
        """{kernel name: (total ms, launches)} since the previous call."""
        ms = np.zeros(K_COUNT, np.float64); n = np.zeros(K_COUNT, np.int64)
        self._check(self.lib.mrf_kernel_times(self.h, ms.ctypes.data, n.ctypes.data))
        return {KERNEL_NAMES[i]: (float(ms[i]), int(n[i])) for i in range(K_COUNT) if n[i]}

    def debug_theta(self):
        inf = self.info()
        W = (inf.n_entries + 31) // 32
        out = np.zeros((inf.n_edge_slots, self.C, W), np.uint32)
        self._check(self.lib.mrf_debug_theta(self.h, out.ctypes.data))
        return out


class mrf_batch_graph_info(ct.Structure):
    _fields_ = [("n_vars", ct.c_int32), ("n_labels", ct.c_int32), ("class_index", ct.c_int32),
                ("site_offset", ct.c_int32), ("first_edge_slot", ct.c_int64)]


BATCH_KEY_STEP = 0x9E3779B97F4A7C15


class MRFBatch:
    """Owner of one mrf_batch_t: many uneven graphs swept together (see mrf.h)."""

    def __init__(self, n_vars, n_labels, n_chains: int, seed: int = 0, use_graphs: bool = True, stream=None,
                 kernel_timing: bool = False, schedule: int = 0):
        lib = load()
        opt = mrf_options()
        lib.mrf_default_options(ct.byref(opt))
        opt.use_graphs = int(use_graphs)
        opt.kernel_timing = int(kernel_timing)
        opt.schedule = int(schedule)
        self.stream = _current_stream() if stream is None else int(stream)
        nv = np.ascontiguousarray(n_vars, np.int32); nl = np.ascontiguousarray(n_labels, np.int32)
        b = _P()
        st = lib.mrf_batch_create(ct.byref(b), nv.shape[0], nv.ctypes.data, nl.ctypes.data, n_chains,
                                  ct.c_uint64(seed & (2**64 - 1)), ct.byref(opt), _P(self.stream))
        if st != MRF_OK:
            raise MrfError(st, lib.mrf_status_string(st).decode())
        self.b, self.lib = b, lib
        self.n_vars, self.n_labels, self.C, self.G = nv, nl, n_chains, nv.shape[0]

    def _check(self, st):
        if st != MRF_OK:
            raise MrfError(st, self.lib.mrf_batch_last_error(self.b).decode())

    def close(self):
        if getattr(self, "b", None):
            self.lib.mrf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_factors(self, models):
        """models: list of workloads.Model in graph order."""
        u = np.ascontiguousarray(np.concatenate([m.unary.ravel() for m in models]), np.float32)
        ne = np.array([m.n_edges for m in models], np.int64)
        s = np.ascontiguousarray(np.concatenate([m.src for m in models]), np.int32)
        t = np.ascontiguousarray(np.concatenate([m.dst for m in models]), np.int32)
        p = np.ascontiguousarray(np.concatenate([m.pair.ravel() for m in models]), np.float32)
        self._check(self.lib.mrf_batch_set_factors(self.b, u.ctypes.data, ne.ctypes.data, s.ctypes.data,
                                                   t.ctypes.data, p.ctypes.data))

    def edit_factors(self, rm_graph, rm_slot, add_graph, src, dst, pair_flat):
        rg = np.ascontiguousarray(rm_graph, np.int32); rs = np.ascontiguousarray(rm_slot, np.int64)
        ag = np.ascontiguousarray(add_graph, np.int32)
        s = np.ascontiguousarray(src, np.int32); t = np.ascontiguousarray(dst, np.int32)
        p = np.ascontiguousarray(pair_flat, np.float32)
        out = np.zeros(ag.shape[0], np.int64)
        self._check(self.lib.mrf_batch_edit_factors(self.b, rg.shape[0], rg.ctypes.data, rs.ctypes.data, ag.shape[0],
                                                    ag.ctypes.data, s.ctypes.data, t.ctypes.data, p.ctypes.data,
                                                    out.ctypes.data))
        return out

    def sweep(self, n: int = 1, mode: int = MODE_PLAIN):
        self._check(self.lib.mrf_batch_sweep(self.b, int(n), int(mode)))

    def set_kernel_timing(self, on: bool):
        """CUDA events around every class kernel (read with class_handle(k).kernel_times())."""
        self._check(self.lib.mrf_batch_set_kernel_timing(self.b, int(bool(on))))

    # -- device edit queue
    def queue_create(self, max_remove: int, max_add: int, max_pair_floats: int, extra_slots: int):
        self._check(self.lib.mrf_batch_queue_create(self.b, int(max_remove), int(max_add), int(max_pair_floats),
                                                    int(extra_slots)))

    def queue_load(self, rm_graph, rm_slot, add_graph, src, dst, pair_flat):
        """Stage the next round's edit: numpy arrays (host) or CUDA tensors
        (device), all of one kind, with the dtypes of mrf_batch_queue_load."""
        dts = (np.int32, np.int64, np.int32, np.int32, np.int32, np.float32)
        arrs = [rm_graph, rm_slot, add_graph, src, dst, pair_flat]
        kinds, ptrs, keep = set(), [], []
        for a, dt in zip(arrs, dts):
            if isinstance(a, np.ndarray) or isinstance(a, (list, tuple)):
                a = np.ascontiguousarray(a, dt)
            else:
                import torch
                if a.dtype != getattr(torch, np.dtype(dt).name):
                    raise TypeError(f"queue_load: expected {np.dtype(dt).name}, got {a.dtype}")
            p, kind, k = _ptr(a)
            kinds.add(kind); ptrs.append(p); keep.append(k)
        if len(kinds) != 1:
            raise TypeError("queue_load: all arrays host or all device")
        n_rm, n_add, n_pair = int(keep[1].shape[0]), int(keep[2].shape[0]), int(keep[5].shape[0])
        if int(keep[0].shape[0]) != n_rm or int(keep[3].shape[0]) != n_add or int(keep[4].shape[0]) != n_add:
            raise ValueError("queue_load: removal or addition arrays of unequal length")
        self._check(self.lib.mrf_batch_queue_load(self.b, n_rm, ptrs[0], ptrs[1], n_add, ptrs[2], ptrs[3], ptrs[4],
                                                  n_pair, ptrs[5], kinds.pop()))
        self._queue_keep = keep                  # host arrays stay alive until the next load

    def round(self, n: int = 10, mode: int = MODE_PLAIN):
        self._check(self.lib.mrf_batch_round(self.b, int(n), int(mode)))

    def queue_result(self, n_add: int):
        """(status bits, class slots of the last round's first n_add additions)."""
        st = ct.c_uint32(0)
        out = np.zeros(int(n_add), np.int64)
        self._check(self.lib.mrf_batch_queue_result(self.b, ct.byref(st), int(n_add), out.ctypes.data if n_add else None))
        return int(st.value), out

    def reset_marginals(self, burn_in: int = 0):
        self._check(self.lib.mrf_batch_reset_marginals(self.b, int(burn_in)))

    def counts(self, g: int):
        out = np.zeros((int(self.n_vars[g]), int(self.n_labels[g])), np.uint32)
        self._check(self.lib.mrf_batch_get_counts(self.b, g, out.ctypes.data))
        return out

    def get_labels(self, g: int):
        out = np.zeros((self.C, int(self.n_vars[g])), np.uint8)
        self._check(self.lib.mrf_batch_get_labels(self.b, g, out.ctypes.data))
        return out

    def graph(self, g: int):
        inf = mrf_batch_graph_info()
        self._check(self.lib.mrf_batch_graph(self.b, g, ct.byref(inf)))
        return inf

    def n_classes(self) -> int:
        return int(self.lib.mrf_batch_n_classes(self.b))

    def class_handle(self, k: int) -> "MRF":
        """A non-owning MRF view of class k (info, kernel times, debug views)."""
        view = MRF.__new__(MRF)
        view.lib = self.lib
        view.h = _P(self.lib.mrf_batch_class(self.b, k))
        view._borrowed = True
        view._batch = self                    # keeps the batch alive while the view is used
        inf = mrf_info()
        self.lib.mrf_get_info(view.h, ct.byref(inf))
        view.N, view.L, view.C = inf.n_vars, inf.n_labels, inf.n_chains
        return view


def philox_rate(threads: int = 152 * 2048 * 8, calls: int = 64, stream: int = 0) -> float:
    """Measured Philox4x32-10 calls per second of a Philox-only kernel."""
    lib = load()
    out = ct.c_double()
    st = lib.mrf_philox_rate(ct.c_uint64(threads), calls, _P(stream), ct.byref(out))
    if st != MRF_OK:
        raise MrfError(st, lib.mrf_status_string(st).decode())
    return out.value


def unpack_theta(words: np.ndarray, m: int) -> np.ndarray:
    """[E][C][W] uint32 -> [C][E][m] bool (bit k of word k // 32)."""
    E, C, W = words.shape
    k = np.arange(m)
    bits = (words[:, :, k // 32] >> (k % 32).astype(np.uint32)) & 1
    return np.transpose(bits.astype(bool), (1, 0, 2))
