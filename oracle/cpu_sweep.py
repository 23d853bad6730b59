"""Python side of oracle/cpu_sweep.c: the primal-dual sweep of Section 5.1 in
float32 on all host cores (OpenMP), for the benchmark's multi-core CPU
baseline.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
legs use this package.  build() compiles the C file with gcc (-O3 -fopenmp)
into oracle/_cpu_sweep.so next to it.

Pin (tests/test_oracle_cpu_sweep.py): one sweep's dual bits and labels equal
those of oracle.sampler.sweep on the same state except draws within 1e-6 of
their decision boundary.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_sweep.c")
LIB = os.path.join(HERE, "_cpu_sweep.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", LIB, SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed for cpu_sweep.c:\n{r.stdout}\n{r.stderr}")
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ct.CDLL(LIB)
        P = ct.c_void_p
        lib.cpu_sweep.restype = ct.c_int
        lib.cpu_sweep.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int64, ct.c_int] + [P] * 15 + \
            [ct.c_uint32, ct.c_uint64, ct.c_int]
        _lib = lib
    return _lib


class CpuSweep:
    """Float32 tables of a decomposition (oracle.decompose) and the site
    incidence, ready for repeated sweeps of C chains."""

    def __init__(self, dec, n_chains: int, seed: int, threads: int = 0):
        self.dec = dec
        self.N, self.L = dec.utilde.shape
        self.E, self.m = dec.ell.shape
        self.C = int(n_chains)
        self.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        self.threads = int(threads)
        f32 = lambda a: np.ascontiguousarray(a, np.float32)
        self.src = np.ascontiguousarray(dec.src, np.int32)
        self.dst = np.ascontiguousarray(dec.dst, np.int32)
        self.q, self.b1, self.b2 = f32(dec.q), f32(dec.beta1), f32(dec.beta2)
        self.active = np.ascontiguousarray(dec.active, np.uint8)
        self.i_pos = np.ascontiguousarray(dec.i_pos, np.int32)
        self.j_pos = np.ascontiguousarray(dec.j_pos, np.int32)
        self.ut = f32(dec.utilde)
        site = np.concatenate([dec.src, dec.dst]).astype(np.int64)
        edge = np.concatenate([np.arange(self.E), np.arange(self.E)]).astype(np.int64)
        side = np.concatenate([np.zeros(self.E, np.uint8), np.ones(self.E, np.uint8)])
        order = np.lexsort((edge, site))
        self.inc_edge = np.ascontiguousarray(edge[order])
        self.inc_side = np.ascontiguousarray(side[order])
        self.inc_ptr = np.zeros(self.N + 1, np.int64)
        np.add.at(self.inc_ptr, site + 1, 1)
        self.inc_ptr = np.cumsum(self.inc_ptr)
        self.W = (self.m + 31) // 32
        self.theta = np.zeros((self.E, self.C, max(1, self.W)), np.uint32)

    def sweep(self, x, sweep_index: int):
        """One sweep from labels x [C][N]; returns the new labels (uint8)."""
        lib = _load()
        xin = np.ascontiguousarray(x, np.uint8)
        xout = np.empty_like(xin)
        p = lambda a: a.ctypes.data
        lib.cpu_sweep(self.N, self.L, self.C, self.E, self.m, p(self.src), p(self.dst), p(self.q), p(self.b1),
                      p(self.b2), p(self.active), p(self.i_pos), p(self.j_pos), p(self.ut), p(self.inc_ptr),
                      p(self.inc_edge), p(self.inc_side), p(xin), p(xout), p(self.theta), int(sweep_index),
                      self.seed, self.threads)
        return xout

    def theta_bits(self):
        """Dual bits of the last sweep as [C][E][m] bool."""
        k = np.arange(self.m)
        bits = (self.theta[:, :, k >> 5] >> (k & 31).astype(np.uint32)) & 1
        return np.transpose(bits, (1, 0, 2)).astype(bool)
