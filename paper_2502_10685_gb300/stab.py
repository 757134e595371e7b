"""Python binding of the C interface (include/stab.h): argument marshalling only.

Every computation runs in libstab.so.  The module exposes the C entry points
under their own names (``stab_create``, ``stab_apply_circuit``, ...) and a
small ``Stab`` class that owns one context, routes its device allocations
through PyTorch's caching allocator and queues its work on a PyTorch stream.

Observables are lists of ``(coeff, string)`` (one letter per qubit, qubit 0
first).  Generator outputs use the library layout index = z | (x << n).
"""
from __future__ import annotations

import ctypes
from typing import Iterable, Optional, Sequence, Tuple

import numpy as np

from . import _lib
from ._lib import (StabBatchItem, StabError, StabGate, StabOpts, StabPathChoice, StabRequest,
                   StabResult, StabServerOpts, StabSparseInfo, StabTerm, check)

KERNELS = {"auto": 0, "resident": 1, "streamed": 2, "plain": 3}
GATE_DTYPE = np.dtype([("op", "u1"), ("q0", "u1"), ("q1", "u1"), ("flags", "u1"),
                       ("param", "<i4")])


def _gates_ptr(gates) -> Tuple[np.ndarray, int]:
    g = np.ascontiguousarray(gates)
    if g.dtype.itemsize != 8 or g.dtype.names is None:
        raise TypeError("gates must be records of the 8-byte stab_gate layout")
    return g, g.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def terms_from_observable(n: int, observable: Iterable[Tuple[float, str]]) -> np.ndarray:
    """[(coeff, "XZIY"...)] -> stab_term records (coeff, x mask, z mask)."""
    obs = list(observable)
    out = np.zeros(len(obs), dtype=[("coeff", "<f8"), ("x", "<u8"), ("z", "<u8")])
    for k, (c, s) in enumerate(obs):
        if len(s) != n:
            raise ValueError("observable string %r has %d letters, expected %d" % (s, len(s), n))
        x = z = 0
        for q, ch in enumerate(s):
            if ch in "XY":
                x |= 1 << q
            if ch in "ZY":
                z |= 1 << q
            if ch not in "IXYZ":
                raise ValueError("bad Pauli letter %r" % ch)
        out[k] = (float(c), x, z)
    return out


# ---------------------------------------------------------------- C names

def stab_default_opts() -> StabOpts:
    o = StabOpts()
    _lib.load().stab_default_opts(ctypes.byref(o))
    return o


def stab_create(n: int, opts: Optional[StabOpts] = None) -> ctypes.c_void_p:
    L = _lib.load()
    h = ctypes.c_void_p()
    check(L.stab_create(n, ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)),
          "stab_create")
    return h


def stab_destroy(h) -> None:
    check(_lib.load().stab_destroy(h), "stab_destroy")


def stab_load_circuit(h, gates, thetas) -> None:
    g, gp = _gates_ptr(gates)
    t = _f64(thetas)
    check(_lib.load().stab_load_circuit(h, gp, g.shape[0], t.ctypes.data if t.size else None,
                                        t.size), "stab_load_circuit")


def stab_set_params(h, thetas, is_device: bool = False) -> None:
    if is_device:
        ptr = thetas.data_ptr()
        check(_lib.load().stab_set_params(h, ptr, 1), "stab_set_params")
    else:
        t = _f64(thetas)
        check(_lib.load().stab_set_params(h, t.ctypes.data if t.size else None, 0),
              "stab_set_params")


def stab_run_generators(h) -> None:
    check(_lib.load().stab_run_generators(h), "stab_run_generators")


def stab_apply_circuit(h, gates, thetas) -> None:
    g, gp = _gates_ptr(gates)
    t = _f64(thetas)
    check(_lib.load().stab_apply_circuit(h, gp, g.shape[0], t.ctypes.data if t.size else None,
                                         t.size), "stab_apply_circuit")


def stab_get_generators(h, n: int, out=None):
    """Host numpy (n, 4^n) by default; a CUDA torch tensor ``out`` is filled on device."""
    if out is None:
        arr = np.empty((n, 4 ** n), dtype=np.float64)
        check(_lib.load().stab_get_generators(h, arr.ctypes.data, 0), "stab_get_generators")
        return arr
    if hasattr(out, "data_ptr"):
        if out.numel() != n * 4 ** n or not out.is_contiguous():
            raise ValueError("out must be a contiguous tensor of n * 4^n doubles")
        check(_lib.load().stab_get_generators(h, out.data_ptr(), 1 if out.is_cuda else 0),
              "stab_get_generators")
        return out
    arr = out
    if arr.dtype != np.float64 or arr.size != n * 4 ** n or not arr.flags.c_contiguous:
        raise ValueError("out must be a contiguous float64 array of n * 4^n entries")
    check(_lib.load().stab_get_generators(h, arr.ctypes.data, 0), "stab_get_generators")
    return arr


def stab_expect(h, terms: np.ndarray) -> float:
    out = ctypes.c_double()
    t = np.ascontiguousarray(terms)
    check(_lib.load().stab_expect(h, t.ctypes.data if t.size else None, t.shape[0],
                                  ctypes.byref(out)), "stab_expect")
    return out.value


def stab_grad(h, terms: np.ndarray, n_params: int) -> Tuple[float, np.ndarray]:
    out = ctypes.c_double()
    grads = np.zeros(max(n_params, 1))
    t = np.ascontiguousarray(terms)
    check(_lib.load().stab_grad(h, t.ctypes.data if t.size else None, t.shape[0],
                                ctypes.byref(out), grads.ctypes.data), "stab_grad")
    return out.value, grads[:n_params]


def stab_set_observable(h, terms: np.ndarray) -> None:
    t = np.ascontiguousarray(terms)
    check(_lib.load().stab_set_observable(h, t.ctypes.data if t.size else None, t.shape[0]),
          "stab_set_observable")


def stab_expect_async(h, out_dev) -> None:
    """``out_dev``: a CUDA float64 tensor (first element receives <O>)."""
    check(_lib.load().stab_expect_async(h, out_dev.data_ptr()), "stab_expect_async")


def stab_grad_async(h, expect_dev, grads_dev) -> None:
    check(_lib.load().stab_grad_async(h, expect_dev.data_ptr() if expect_dev is not None else None,
                                      grads_dev.data_ptr()), "stab_grad_async")


def stab_transfer_bytes(h) -> Tuple[int, int]:
    a, b = ctypes.c_int64(), ctypes.c_int64()
    check(_lib.load().stab_transfer_bytes(h, ctypes.byref(a), ctypes.byref(b)),
          "stab_transfer_bytes")
    return a.value, b.value


def stab_synchronize(h) -> None:
    check(_lib.load().stab_synchronize(h), "stab_synchronize")


def stab_plan_info(h) -> Tuple[int, int, int]:
    a, b, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    check(_lib.load().stab_plan_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k)),
          "stab_plan_info")
    return a.value, b.value, k.value


def stab_split_info(h) -> Tuple[int, int, int]:
    """(cut, generator units, expectation units) of the split sweeps; cut -1: none."""
    a, g, e = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    check(_lib.load().stab_split_info(h, ctypes.byref(a), ctypes.byref(g), ctypes.byref(e)),
          "stab_split_info")
    return a.value, g.value, e.value


def stab_launch_count(h) -> int:
    return int(_lib.load().stab_launch_count(h))


# ---------------------------------------------------------------- class

def stab_probe_fp64(kind: str = "dfma", iters: int = 8192) -> Tuple[float, float]:
    """FP64 rate of the current device: (TFLOP/s, ms of the timed launch);
    kind "dfma" (independent DFMA chains) or "dmma" (8x8x4 FP64 matrix
    instruction chains)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    check(_lib.load().stab_probe_fp64({"dfma": 0, "dmma": 1}[kind], int(iters),
                                      ctypes.byref(tf), ctypes.byref(ms)), "stab_probe_fp64")
    return tf.value, ms.value


def stab_probe_pass(pattern: int, threads: int = 256, passes: int = 40000) -> float:
    """Cycles per pass of the n = 4 register pass loop's pieces on one CTA:
    pattern 0 register passes, 1 + a layout switch every second pass, 2 + a
    four-CNOT pull every fourth, 3 two entries per thread and one barrier per
    four passes (threads = 128), 4 two-wire fused passes (cycles per wire
    pass, two per fused pass)."""
    clk = ctypes.c_double()
    check(_lib.load().stab_probe_pass(int(pattern), int(threads), int(passes),
                                      ctypes.byref(clk)), "stab_probe_pass")
    return clk.value


def _choice_dict(c: StabPathChoice) -> dict:
    return {"resident": c.resident, "resident_adjoint": c.resident_adjoint,
            "gen_cut": c.gen_cut, "tile_limit": c.tile_limit, "tuned": c.tuned,
            "gen_parts": c.gen_parts}


def stab_path_tune(device: int, n: int) -> dict:
    """Measures the path choices for n qubits on `device` now (and caches them)."""
    c = StabPathChoice()
    check(_lib.load().stab_path_tune(device, n, ctypes.byref(c)), "stab_path_tune")
    return _choice_dict(c)


def stab_path_lookup(gpu_name: str, n: int) -> Optional[dict]:
    c = StabPathChoice()
    rc = _lib.load().stab_path_lookup(gpu_name.encode(), n, ctypes.byref(c))
    if rc == -7:
        return None
    check(rc, "stab_path_lookup")
    return _choice_dict(c)


def stab_path_store(gpu_name: str, n: int, choice: dict) -> None:
    c = StabPathChoice(**{k: choice[k] for k in ("resident", "resident_adjoint", "gen_cut",
                                                  "tile_limit", "tuned")})
    c.gen_parts = int(choice.get("gen_parts", 2))
    check(_lib.load().stab_path_store(gpu_name.encode(), n, ctypes.byref(c)), "stab_path_store")


class Stab:
    """One context: n qubits, a loaded circuit, its generators and observables.

    ``torch_memory=True`` routes device allocations through PyTorch's caching
    allocator and queues work on the current PyTorch stream of ``device``.
    """

    def __init__(self, n: int, kernel: str = "auto", fuse: bool = True, device: int = 0,
                 torch_memory: bool = True, stream=None):
        self.n = n
        self.n_params = 0
        self._keep = []
        opts = stab_default_opts()
        opts.device = device
        opts.kernel = KERNELS[kernel]
        opts.fuse = 1 if fuse else 0
        if torch_memory or stream is not None:
            import torch
            dev = torch.device("cuda", device)
            if stream is None:
                stream = torch.cuda.current_stream(dev)
            opts.stream = ctypes.c_void_p(stream.cuda_stream)
            opts.stream_given = 1
            self._stream = stream
        if torch_memory:
            import torch

            def _alloc(nbytes, st, user):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), device,
                                                                  self._stream))
                except Exception:
                    return None

            def _free(ptr, nbytes, st, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            a, f = _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)
            self._keep += [a, f]
            opts.alloc = a
            opts.free = f
        self.h = stab_create(n, opts)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            stab_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_circuit(self, gates, thetas) -> None:
        stab_load_circuit(self.h, gates, thetas)
        self.n_params = int(np.asarray(thetas).size)

    def set_params(self, thetas) -> None:
        if hasattr(thetas, "is_cuda") and thetas.is_cuda:
            import torch
            t = thetas.detach().to(torch.float64).contiguous()
            if t.numel() != self.n_params:
                raise ValueError("expected %d angles" % self.n_params)
            stab_set_params(self.h, t, True)
            self._keep_params = t
        else:
            t = np.asarray(thetas.detach().cpu() if hasattr(thetas, "detach") else thetas,
                           dtype=np.float64)
            if t.size != self.n_params:
                raise ValueError("expected %d angles" % self.n_params)
            stab_set_params(self.h, t, False)

    def run_generators(self) -> None:
        stab_run_generators(self.h)

    def apply_circuit(self, gates, thetas) -> None:
        stab_apply_circuit(self.h, gates, thetas)
        self.n_params = int(np.asarray(thetas).size)

    def generators(self, out=None):
        return stab_get_generators(self.h, self.n, out)

    def expect(self, observable) -> float:
        return stab_expect(self.h, terms_from_observable(self.n, observable))

    def grad(self, observable) -> Tuple[float, np.ndarray]:
        return stab_grad(self.h, terms_from_observable(self.n, observable), self.n_params)

    def set_observable(self, observable) -> None:
        stab_set_observable(self.h, terms_from_observable(self.n, observable))

    def expect_async(self, out_dev) -> None:
        stab_expect_async(self.h, out_dev)

    def grad_async(self, expect_dev, grads_dev) -> None:
        stab_grad_async(self.h, expect_dev, grads_dev)

    def transfer_bytes(self):
        return stab_transfer_bytes(self.h)

    def density_matrix(self) -> np.ndarray:
        """rho of U|0^n>, complex (2^n, 2^n); row/column bit q is qubit q."""
        D = 2 ** self.n
        out = np.empty((D, D), dtype=np.complex128)
        check(_lib.load().stab_density_matrix(self.h, out.ctypes.data, 0), "stab_density_matrix")
        return out

    def synchronize(self) -> None:
        stab_synchronize(self.h)

    def plan_info(self):
        return stab_plan_info(self.h)

    def split_info(self):
        return stab_split_info(self.h)

    def launch_count(self) -> int:
        return stab_launch_count(self.h)

    def grad_parts(self) -> int:
        """K >= 2: the last gradient was cut into the generators' K parts;
        1: meet-in-the-middle or streamed; 0: no gradient since the load."""
        k = ctypes.c_int32()
        check(_lib.load().stab_grad_parts(self.h, ctypes.byref(k)), "stab_grad_parts")
        return k.value

    def path_choice(self) -> dict:
        """The path this context runs with (the tuner's choice for AUTO)."""
        c = StabPathChoice()
        check(_lib.load().stab_path_current(self.h, ctypes.byref(c)), "stab_path_current")
        return _choice_dict(c)


# ---------------------------------------------------------------- batches

ITEM_KINDS = {"generators": 0, "expect": 1}


def _torch_alloc_opts(opts, device, holder):
    import torch
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    opts.stream = ctypes.c_void_p(stream.cuda_stream)
    opts.stream_given = 1

    def _alloc(nbytes, st, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream))
        except Exception:
            return None

    def _free(ptr, nbytes, st, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)
    holder += [a, f, stream]
    opts.alloc = a
    opts.free = f


class Batch:
    """Many uneven circuits evaluated by one persistent launch.

    ``items``: objects with ``circuit`` (workloads.Circuit), ``kind``
    ("generators" or "expect") and ``observable`` (for "expect").
    """

    def __init__(self, items, device: int = 0, kernel: str = "auto", torch_memory: bool = True):
        self._keep = []
        self.items = list(items)
        arr = (StabBatchItem * len(self.items))()
        for k, it in enumerate(self.items):
            c = it.circuit
            g = np.ascontiguousarray(c.gates)
            th = np.ascontiguousarray(c.thetas if c.n_params else np.zeros(1), dtype=np.float64)
            self._keep += [g, th]
            arr[k].n = c.n
            arr[k].kind = ITEM_KINDS[it.kind]
            arr[k].gates = g.ctypes.data if c.m else None
            arr[k].m = c.m
            arr[k].thetas = th.ctypes.data
            arr[k].n_params = c.n_params
            if it.kind == "expect":
                t = terms_from_observable(c.n, it.observable)
                self._keep.append(t)
                arr[k].obs = t.ctypes.data if len(t) else None
                arr[k].n_terms = len(t)
        opts = stab_default_opts()
        opts.device = device
        opts.kernel = KERNELS[kernel]
        if torch_memory:
            _torch_alloc_opts(opts, device, self._keep)
        h = ctypes.c_void_p()
        check(_lib.load().stab_batch_create(arr, len(self.items), ctypes.byref(opts),
                                            ctypes.byref(h)), "stab_batch_create")
        self.h = h
        self._keep = [x for x in self._keep if not isinstance(x, np.ndarray)]

    def run(self) -> None:
        check(_lib.load().stab_apply_batch(self.h), "stab_apply_batch")

    def expectations(self) -> np.ndarray:
        out = np.empty(len(self.items))
        check(_lib.load().stab_batch_expectations(self.h, out.ctypes.data),
              "stab_batch_expectations")
        return out

    def generators(self, item: int) -> np.ndarray:
        n = self.items[item].circuit.n
        out = np.empty((n, 4 ** n))
        check(_lib.load().stab_batch_generators(self.h, item, out.ctypes.data, 0),
              "stab_batch_generators")
        return out

    def info(self):
        u, g, o, sn = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(_lib.load().stab_batch_info(self.h, ctypes.byref(u), ctypes.byref(g),
                                          ctypes.byref(o), ctypes.byref(sn)), "stab_batch_info")
        return {"units": u.value, "grid": g.value, "ctas_per_sm": o.value,
                "smem_max_n": sn.value}

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            _lib.load().stab_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- sparse term lists

TERM_DTYPE = np.dtype([("coeff", "<f8"), ("x", "<u8"), ("z", "<u8")])


def _info_dict(info: StabSparseInfo) -> dict:
    return {"order_final": info.order_final, "order_max": info.order_max, "steps": info.steps,
            "dense_gates": info.dense_gates, "regrows": info.regrows}


class Sparse:
    """A stabilizer or observable held as its list of Pauli terms (stab_sparse_*),
    for up to 32 qubits while the stabilizer order stays below ``max_terms``.

    ``expect`` returns ``(value, info)``; ``generator`` returns the term records
    (``coeff``, ``x``, ``z`` masks, bit q = qubit q) and ``info``.  With
    ``torch_memory`` the device buffers come from PyTorch's caching allocator
    and the work is queued on its current stream.
    """

    def __init__(self, n: int, max_terms: int = 1 << 24, device: int = 0,
                 torch_memory: bool = True):
        self.n = n
        self._keep = []
        o = StabOpts()
        _lib.load().stab_default_opts(ctypes.byref(o))
        o.device = device
        if torch_memory:
            _torch_alloc_opts(o, device, self._keep)
        h = ctypes.c_void_p()
        check(_lib.load().stab_sparse_create(n, int(max_terms), ctypes.byref(o), ctypes.byref(h)),
              "stab_sparse_create")
        self.h = h

    def load_circuit(self, gates, thetas) -> None:
        g, gp = _gates_ptr(gates)
        m = int(g.shape[0])
        th = _f64(thetas)
        self._n_params = int(th.size)
        check(_lib.load().stab_sparse_load_circuit(self.h, gp if m else None, m,
                                                   th.ctypes.data if th.size else None, th.size),
              "stab_sparse_load_circuit")

    def set_dense_threshold(self, order: int) -> None:
        check(_lib.load().stab_sparse_set_dense_threshold(self.h, int(order)),
              "stab_sparse_set_dense_threshold")

    def expect(self, observable):
        t = terms_from_observable(self.n, observable)
        out = ctypes.c_double()
        info = StabSparseInfo()
        check(_lib.load().stab_sparse_expect(self.h, t.ctypes.data if len(t) else None, len(t),
                                             ctypes.byref(out), ctypes.byref(info)),
              "stab_sparse_expect")
        return out.value, _info_dict(info)

    def generator(self, k: int, max_out: int = 1 << 22):
        out = np.zeros(max(1, max_out), dtype=TERM_DTYPE)
        cnt = ctypes.c_int64()
        info = StabSparseInfo()
        check(_lib.load().stab_sparse_generator(self.h, k, max_out, out.ctypes.data,
                                                ctypes.byref(cnt), ctypes.byref(info)),
              "stab_sparse_generator")
        return out[:cnt.value].copy(), _info_dict(info)

    def order_history(self) -> np.ndarray:
        cnt = ctypes.c_int64()
        check(_lib.load().stab_sparse_order_history(self.h, None, 0, ctypes.byref(cnt)),
              "stab_sparse_order_history")
        out = np.zeros(max(1, cnt.value), dtype=np.int64)
        check(_lib.load().stab_sparse_order_history(self.h, out.ctypes.data, cnt.value,
                                                    ctypes.byref(cnt)),
              "stab_sparse_order_history")
        return out[:cnt.value]

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            _lib.load().stab_sparse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving

REQUEST_KINDS = {"expect": 0, "grad": 1}


class Server:
    """Continuous-batching request server (stab_server_*).

    ``submit`` copies the request and returns its id immediately; ``wait``
    blocks for its result: a dict with ``status``, ``expect``, ``grads`` (for
    gradient requests) and the server-clock times ``submit_s``, ``admit_s``,
    ``done_s``.
    """

    POLICIES = {"fifo": 0, "shortest": 1}
    ENGINES = {"iterate": 0, "contexts": 1}

    def __init__(self, device: int = 0, max_active: int = 0, hbm_budget: int = 0,
                 planners: int = 0, policy: str = "fifo", engine: str = "iterate",
                 iter_chunks: int = 0, iter_smem_kb: int = 0, iter_max_n: int = 0,
                 iter_slice_us: float = 0.0, aging_s: float = 0.0, torch_memory: bool = True):
        o = StabServerOpts()
        o.device = device
        o.max_active = max_active
        o.hbm_budget = hbm_budget
        o.planners = planners
        o.policy = self.POLICIES[policy]
        o.engine = self.ENGINES[engine]
        o.iter_chunks = iter_chunks
        o.iter_smem_kb = iter_smem_kb
        o.iter_max_n = iter_max_n
        o.iter_slice_us = iter_slice_us
        o.aging_s = aging_s
        self._keep = []
        if torch_memory:
            # device memory of the server's requests and contexts from
            # PyTorch's caching allocator; the library hands a block back only
            # after the work that used it has completed
            import torch

            def _alloc(nbytes, st, user):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), device))
                except Exception:
                    return None

            def _free(ptr, nbytes, st, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            a, f = _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)
            self._keep += [a, f]
            o.alloc = a
            o.free = f
        h = ctypes.c_void_p()
        check(_lib.load().stab_server_create(ctypes.byref(o), ctypes.byref(h)),
              "stab_server_create")
        self.h = h
        self._n_params = {}

    @staticmethod
    def _request(circuit, kind, observable, keep):
        r = StabRequest()
        g = np.ascontiguousarray(circuit.gates)
        th = np.ascontiguousarray(circuit.thetas if circuit.n_params else np.zeros(1),
                                  dtype=np.float64)
        t = terms_from_observable(circuit.n, observable)
        keep += [g, th, t]
        r.n = circuit.n
        r.kind = REQUEST_KINDS[kind]
        r.gates = g.ctypes.data if circuit.m else None
        r.m = circuit.m
        r.thetas = th.ctypes.data
        r.n_params = circuit.n_params
        r.obs = t.ctypes.data if len(t) else None
        r.n_terms = len(t)
        return r

    @staticmethod
    def footprint(circuit, kind: str, observable) -> int:
        keep = []
        r = Server._request(circuit, kind, observable, keep)
        return int(_lib.load().stab_request_footprint(ctypes.byref(r)))

    def submit(self, circuit, kind: str, observable) -> int:
        keep = []
        r = self._request(circuit, kind, observable, keep)
        i = ctypes.c_int64()
        check(_lib.load().stab_server_submit(self.h, ctypes.byref(r), ctypes.byref(i)),
              "stab_server_submit")
        self._n_params[i.value] = circuit.n_params
        return i.value

    def wait(self, rid: int, timeout_s: float = -1.0) -> dict:
        res = StabResult()
        npar = self._n_params.get(rid, 0)
        grads = np.zeros(max(npar, 1))
        check(_lib.load().stab_server_wait(self.h, rid, timeout_s, ctypes.byref(res),
                                           grads.ctypes.data), "stab_server_wait")
        return {"status": res.status, "expect": res.expect, "grads": grads[:npar],
                "submit_s": res.submit_s, "admit_s": res.admit_s, "done_s": res.done_s}

    def done(self, rid: int) -> bool:
        d = ctypes.c_int32()
        check(_lib.load().stab_server_poll(self.h, rid, ctypes.byref(d)), "stab_server_poll")
        return bool(d.value)

    def stats(self) -> dict:
        a, b, c, d = (ctypes.c_int64() for _ in range(4))
        check(_lib.load().stab_server_stats(self.h, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c), ctypes.byref(d)), "stab_server_stats")
        return {"submitted": a.value, "completed": b.value, "active": c.value,
                "bytes_in_use": d.value}

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            _lib.load().stab_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
