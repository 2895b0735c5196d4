"""Python binding of the DUWP CUDA library (libduwp.so, C ABI in include/duwp.h).

Argument marshalling only: every step of the method runs in the library's kernels.  PyTorch
provides device memory (the caching allocator is handed to the library as its allocator
callbacks) and the CUDA stream.  There is no CPU fallback: without the compiled library or a
CUDA device every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libduwp.so")

OK, EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, EBUSY, EOVERFLOW, ENOTFOUND, PENDING = 0, -1, -2, -3, -4, -5, -6, -7, -8, 1
INSTANT, AVERAGED = 0, 1
BC = {"inout": 0, "specular": 1, "periodic": 2, "vacuum": 3}
PRECISION = {"fp64": 0, "fp32": 1}
EPS = {"eps1": 0, "eps12": 1, "eps0": 2, "eps_avg": 3}
FLUX = {"gks_eq": 0, "kfvs": 1}
NTC = {"particle": 0, "total": 1}
RESAMPLE = {"maxwell": 0, "ce": 1}
SPLIT = {"p": 0, "qmc": 1}
RECON = {"first": 0, "vanleer": 1}

# Every symbol of include/duwp.h (checked by the CPU test-suite against the built library).
EXPORTS = (
    "duwp_init", "duwp_init_batch", "duwp_step", "duwp_sync", "duwp_step_timed", "duwp_moments", "duwp_moments_all", "duwp_moments_all_async", "duwp_moments_wait", "duwp_fields", "duwp_get_info",
    "duwp_destroy", "duwp_error_string", "duwp_last_cuda_error", "duwp_set_launch", "duwp_use_graphs",
    "duwp_num_particles", "duwp_get_particles", "duwp_get_counters", "duwp_get_cmax", "duwp_checkpoint_size",
    "duwp_checkpoint_save", "duwp_checkpoint_restore", "duwp_server_create", "duwp_submit", "duwp_poll",
    "duwp_server_destroy", "duwp_get_particles_noalloc", "duwp_stress_heat", "duwp_stress_heat_accumulate",
    "duwp_split_create", "duwp_split_step", "duwp_split_part", "duwp_split_destroy", "duwp_shock_normalise",
)


class DuwpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {_error_string(status)} ({status})"
        if status == ECUDA and _lib is not None:
            msg += ": " + _lib.duwp_last_cuda_error().decode()
        super().__init__(msg)


class State(C.Structure):
    _fields_ = [("rho", C.c_double), ("u", C.c_double), ("v", C.c_double), ("w", C.c_double), ("T", C.c_double)]


class Params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("Pr", C.c_double), ("R", C.c_double),
        ("omega", C.c_double), ("alpha", C.c_double),
        ("rho_ref", C.c_double), ("T_ref", C.c_double), ("Kn", C.c_double), ("L_ref", C.c_double),
        ("x_min", C.c_double), ("x_max", C.c_double),
        ("n_cells", C.c_int32),
        ("dt", C.c_double), ("cfl", C.c_double),
        ("left", State), ("right", State),
        ("x_split", C.c_double),
        ("bc_left", C.c_int32), ("bc_right", C.c_int32),
        ("ppc_ref", C.c_double),
        ("precision", C.c_int32), ("eps_mode", C.c_int32), ("flux_mode", C.c_int32), ("ntc_rate", C.c_int32),
        ("seed", C.c_uint64),
        ("capacity", C.c_uint64),
        ("avg_start", C.c_int32),
        ("resample_mode", C.c_int32),
        ("split_mode", C.c_int32),
        ("recon_mode", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [("dx", C.c_double), ("dt", C.c_double), ("mp", C.c_double), ("beta", C.c_double),
                ("lambda_ref", C.c_double), ("mu_ref", C.c_double), ("c_ref", C.c_double),
                ("capacity", C.c_int64), ("n_instances", C.c_int32),
                ("steps_done", C.c_int64), ("particle_updates", C.c_int64)]


class ServerCfg(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_slots", C.c_int32), ("max_cells", C.c_int32),
                ("steps_per_launch", C.c_int32), ("precision", C.c_int32), ("stream", C.c_void_p),
                ("lanes", C.c_int32), ("long_steps", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_cells", C.c_int32), ("steps", C.c_int64),
                ("particle_updates", C.c_int64), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("step_p50_ms", C.c_double), ("step_p99_ms", C.c_double),
                ("rho", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_double)), ("T", C.POINTER(C.c_double))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None
_lock = threading.Lock()


def _error_string(status: int) -> str:
    if _lib is None:
        return "status"
    return _lib.duwp_error_string(status).decode()


def load(path: str = LIB_PATH):
    """Load libduwp.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"DUWP CUDA library not built ({path}); run paper_2305_12071_gb300.build.build()")
        L = C.CDLL(path)
        i32, i64, u64, vp, dp = C.c_int32, C.c_int64, C.c_uint64, C.c_void_p, C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        L.duwp_error_string.restype = C.c_char_p
        L.duwp_error_string.argtypes = [C.c_int]
        L.duwp_last_cuda_error.restype = C.c_char_p
        L.duwp_init.argtypes = [C.POINTER(Params), vp, ALLOC_FN, FREE_FN, vp, C.POINTER(vp)]
        L.duwp_init_batch.argtypes = [C.POINTER(Params), i32, vp, ALLOC_FN, FREE_FN, vp, C.POINTER(vp)]
        L.duwp_step.argtypes = [vp, i32]
        L.duwp_sync.argtypes = [vp]
        L.duwp_step_timed.argtypes = [vp, i32, dp, dp]
        L.duwp_moments.argtypes = [vp, i32, i32, dp, dp, dp, dp, i32]
        L.duwp_moments_all.argtypes = [vp, i32, dp, dp, dp, dp, i64]
        L.duwp_moments_all_async.argtypes = [vp, i32, dp, dp, dp, dp, i64]
        L.duwp_moments_wait.argtypes = [vp]
        L.duwp_stress_heat.argtypes = [vp, i32, i32, dp, dp, i32]
        L.duwp_stress_heat_accumulate.argtypes = [vp]
        L.duwp_fields.argtypes = [vp, i32, i32, dp, i32, C.POINTER(i64)]
        L.duwp_get_info.argtypes = [vp, i32, C.POINTER(Info)]
        L.duwp_destroy.argtypes = [vp]
        L.duwp_set_launch.argtypes = [vp, i32, i32, i32]
        L.duwp_use_graphs.argtypes = [vp, i32]
        L.duwp_num_particles.argtypes = [vp, i32, C.POINTER(i64)]
        L.duwp_get_particles.argtypes = [vp, i32, ip, dp, dp, dp, dp, i64]
        L.duwp_get_counters.argtypes = [vp, i32, ip, ip, ip, ip, i32]
        L.duwp_get_particles_noalloc.argtypes = [vp, i32, vp, vp, vp, vp, vp, i64]
        L.duwp_get_cmax.argtypes = [vp, i32, dp, i32]
        L.duwp_checkpoint_size.argtypes = [vp, C.POINTER(u64)]
        L.duwp_checkpoint_save.argtypes = [vp, vp, u64]
        L.duwp_checkpoint_restore.argtypes = [vp, vp, u64]
        L.duwp_server_create.argtypes = [C.POINTER(ServerCfg), ALLOC_FN, FREE_FN, vp, C.POINTER(vp)]
        L.duwp_submit.argtypes = [vp, C.POINTER(Params), i32, C.POINTER(u64)]
        L.duwp_poll.argtypes = [vp, u64, C.POINTER(Result)]
        L.duwp_server_destroy.argtypes = [vp]
        L.duwp_split_create.argtypes = [C.POINTER(Params), i32, ip, ALLOC_FN, FREE_FN, vp, C.POINTER(vp)]
        L.duwp_split_step.argtypes = [vp, i32]
        L.duwp_split_part.argtypes = [vp, i32, C.POINTER(vp), ip, ip]
        L.duwp_split_destroy.argtypes = [vp]
        L.duwp_shock_normalise.argtypes = [i32, i64, dp, dp, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                           C.c_double, C.c_double, C.c_double, C.c_double, dp, dp, dp, dp, dp]
        _lib = L
        return L


def make_params(p: dict) -> Params:
    """Marshal a problem dict (see paper_2305_12071_gb300.workloads) into duwp_params."""
    s = Params()
    s.gamma = p.get("gamma", 5.0 / 3.0)
    s.Pr = p.get("Pr", 2.0 / 3.0)
    s.R = p.get("R", 1.0)
    s.omega = p["omega"]
    s.alpha = p.get("alpha", 1.0)
    s.rho_ref = p.get("rho_ref", 1.0)
    s.T_ref = p.get("T_ref", 1.0)
    s.Kn = p["Kn"]
    s.L_ref = p.get("L_ref", 1.0)
    s.x_min, s.x_max = p["x_min"], p["x_max"]
    s.n_cells = int(p["n_cells"])
    s.dt = p.get("dt", 0.0)
    s.cfl = p.get("cfl", 0.5)
    s.left = State(*p["left"])
    s.right = State(*p["right"])
    s.x_split = p.get("x_split", 0.5 * (p["x_min"] + p["x_max"]))
    s.bc_left = BC[p.get("bc_left", "inout")]
    s.bc_right = BC[p.get("bc_right", "inout")]
    s.ppc_ref = p["ppc_ref"]
    s.precision = PRECISION[p.get("precision", "fp64")]
    s.eps_mode = EPS[p.get("eps_mode", "eps1")]
    s.flux_mode = FLUX[p.get("flux_mode", "gks_eq")]
    s.ntc_rate = NTC[p.get("ntc_rate", "particle")]
    s.seed = int(p.get("seed", 1)) & 0xFFFFFFFFFFFFFFFF
    s.capacity = int(p.get("capacity", 0))
    s.avg_start = int(p.get("avg_start", 0))
    s.resample_mode = RESAMPLE[p.get("resample_mode", "maxwell")]
    s.split_mode = SPLIT[p.get("split_mode", "p")]
    s.recon_mode = RECON[p.get("recon_mode", "first")]
    return s


class _TorchAllocator:
    """Allocator callbacks backed by torch's CUDA caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device
        self.calls = 0          # allocations requested by the library so far
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
        except Exception:
            return None

    def _free(self, ptr, nbytes, stream, ctx):
        if ptr:
            self.torch.cuda.caching_allocator_delete(int(ptr))


def _chk(rc: int, where: str):
    if rc != OK:
        raise DuwpError(rc, where)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class Solver:
    """One handle of the library: a single instance or a batch stepped together.

    params: a problem dict or a list of them (one precision for all).  The handle owns its own
    CUDA stream (a torch stream) so its steps can be captured in CUDA graphs."""

    def __init__(self, params, device: int = 0, torch_alloc: bool = True, graphs: bool = True):
        import torch
        L = load()
        if not torch.cuda.is_available():
            raise RuntimeError("the DUWP library needs a CUDA device")
        plist = [params] if isinstance(params, dict) else list(params)
        self.params = plist
        self.n = len(plist)
        torch.cuda.set_device(device)
        self.stream = torch.cuda.Stream(device=device)
        arr = (Params * self.n)(*[make_params(p) for p in plist])
        self._alloc = _TorchAllocator(device) if torch_alloc else None
        h = C.c_void_p()
        a = self._alloc.alloc if self._alloc else ALLOC_FN()
        f = self._alloc.free if self._alloc else FREE_FN()
        _chk(L.duwp_init_batch(arr, self.n, C.c_void_p(self.stream.cuda_stream), a, f, None, C.byref(h)),
             "duwp_init_batch")
        self.h = h
        self.L = L
        if not graphs:
            _chk(L.duwp_use_graphs(self.h, 0), "duwp_use_graphs")

    def close(self):
        if getattr(self, "h", None):
            self.L.duwp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        _chk(self.L.duwp_step(self.h, int(n)), "duwp_step")

    def sync(self):
        _chk(self.L.duwp_sync(self.h), "duwp_sync")

    KERNELS = ("k_collide", "k_stream", "k_far_sort", "k_cells", "k_offsets_flux")
    TIMED_SLOTS = 7
    # slot of each kernel in step_timed's kernel_ms (slot 5: the span of all steps)
    KERNEL_SLOTS = {"k_staged": 6, "k_collide": 0, "k_stream": 1, "k_far_sort": 2, "k_cells": 3, "k_offsets_flux": 4}

    def step_timed(self, n: int):
        """n steps as plain launches with CUDA events around each kernel: returns (kernel_ms[7]: summed
        over the steps for the kernels named in KERNELS, then the span of all n steps, then the
        staged-cell kernel k_staged; per-step ms)."""
        k = np.zeros(self.TIMED_SLOTS, np.float64)
        st = np.zeros(int(n), np.float64)
        _chk(self.L.duwp_step_timed(self.h, int(n), _dptr(k), _dptr(st)), "duwp_step_timed")
        return k, st

    def particle_updates(self) -> int:
        return int(sum(self.info(i)["particle_updates"] for i in range(self.n)))

    def use_graphs(self, on: bool):
        _chk(self.L.duwp_use_graphs(self.h, 1 if on else 0), "duwp_use_graphs")

    def set_launch(self, threads: int, reg_capped: int = 0, groups: int = 2):
        _chk(self.L.duwp_set_launch(self.h, int(threads), int(reg_capped), int(groups)), "duwp_set_launch")

    def n_cells(self, inst: int = 0) -> int:
        return int(self.params[inst]["n_cells"])

    def info(self, inst: int = 0) -> dict:
        o = Info()
        _chk(self.L.duwp_get_info(self.h, inst, C.byref(o)), "duwp_get_info")
        return {k: getattr(o, k) for k, _ in Info._fields_}

    def fields(self, inst: int = 0, which: int = INSTANT):
        n = self.n_cells(inst)
        out = np.empty((n, 5), np.float64)
        navg = C.c_int64()
        _chk(self.L.duwp_fields(self.h, inst, which, _dptr(out), n, C.byref(navg)), "duwp_fields")
        return out, int(navg.value)

    def moments(self, inst: int = 0, which: int = INSTANT) -> dict:
        n = self.n_cells(inst)
        r, u, T, wf = (np.empty(n, np.float64) for _ in range(4))
        _chk(self.L.duwp_moments(self.h, inst, which, _dptr(r), _dptr(u), _dptr(T), _dptr(wf), n), "duwp_moments")
        return {"rho": r, "u": u, "T": T, "wave_frac": wf}

    def stress_heat(self, inst: int = 0, which: int = INSTANT) -> dict:
        """Normal stress Pi = S_xx and heat flux Q = Q_x per cell (Eq. gkt_moment1) of the current
        state, or (AVERAGED) the mean of the states taken by stress_heat_accumulate."""
        n = self.n_cells(inst)
        Pi, Q = np.empty(n, np.float64), np.empty(n, np.float64)
        _chk(self.L.duwp_stress_heat(self.h, inst, which, _dptr(Pi), _dptr(Q), n), "duwp_stress_heat")
        return {"Pi": Pi, "Q": Q}

    def stress_heat_accumulate(self):
        """Adds the current Pi and Q of every cell to the running sums (enqueued, non-blocking)."""
        _chk(self.L.duwp_stress_heat_accumulate(self.h), "duwp_stress_heat_accumulate")

    def moments_all(self, which: int = INSTANT, out: dict | None = None) -> dict:
        """Profiles of every instance at once (concatenated in instance order): one call, one copy.
        `out` (optional) supplies the host arrays to fill (e.g. pinned ones) and is returned."""
        total = sum(self.n_cells(i) for i in range(self.n))
        if out is None:
            out = {k: np.empty(total, np.float64) for k in ("rho", "u", "T", "wave_frac")}
        _chk(self.L.duwp_moments_all(self.h, which, _dptr(out["rho"]), _dptr(out["u"]), _dptr(out["T"]),
                                     _dptr(out["wave_frac"]), total), "duwp_moments_all")
        return out

    def moments_all_async(self, out: dict, which: int = INSTANT) -> dict:
        """Enqueue moments_all into the host arrays of `out` (pinned, so that the copies overlap with
        the next steps) and return at once; the arrays are valid after moments_wait()."""
        total = sum(self.n_cells(i) for i in range(self.n))
        for k in ("rho", "u", "T", "wave_frac"):
            a = out[k]
            if a.shape != (total,) or a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError(f"moments_all_async: out[{k!r}] must hold {total} contiguous float64")
        _chk(self.L.duwp_moments_all_async(self.h, which, _dptr(out["rho"]), _dptr(out["u"]), _dptr(out["T"]),
                                           _dptr(out["wave_frac"]), total), "duwp_moments_all_async")
        return out

    def moments_wait(self):
        _chk(self.L.duwp_moments_wait(self.h), "duwp_moments_wait")

    def num_particles(self, inst: int = 0) -> int:
        o = C.c_int64()
        _chk(self.L.duwp_num_particles(self.h, inst, C.byref(o)), "duwp_num_particles")
        return int(o.value)

    def particles(self, inst: int = 0) -> dict:
        n = self.num_particles(inst)
        cell = np.empty(n, np.int32)
        xl, u, v, w = (np.empty(n, np.float64) for _ in range(4))
        _chk(self.L.duwp_get_particles(self.h, inst, _iptr(cell), _dptr(xl), _dptr(u), _dptr(v), _dptr(w), n),
             "duwp_get_particles")
        return {"cell": cell, "xl": xl, "u": u, "v": v, "w": w}

    def particles_noalloc(self, out: dict, inst: int = 0):
        """Write the particles into caller-owned CUDA tensors (keys cell (int32), xl, u, v, w (float64),
        each of num_particles entries) without any allocation inside the library; asynchronous on the
        handle's stream (call sync() before reading them)."""
        n = int(out["cell"].numel())
        ptr = [C.c_void_p(out[k].data_ptr()) for k in ("cell", "xl", "u", "v", "w")]
        _chk(self.L.duwp_get_particles_noalloc(self.h, inst, *ptr, n), "duwp_get_particles_noalloc")

    def counters(self, inst: int = 0) -> dict:
        n = self.n_cells(inst)
        out = {k: np.empty(n, np.int32) for k in ("ncand", "nacc", "nabs", "nnew")}
        _chk(self.L.duwp_get_counters(self.h, inst, *[_iptr(out[k]) for k in ("ncand", "nacc", "nabs", "nnew")], n),
             "duwp_get_counters")
        return out

    def cmax(self, inst: int = 0) -> np.ndarray:
        n = self.n_cells(inst)
        out = np.empty(n, np.float64)
        _chk(self.L.duwp_get_cmax(self.h, inst, _dptr(out), n), "duwp_get_cmax")
        return out

    def checkpoint(self) -> bytes:
        nb = C.c_uint64()
        _chk(self.L.duwp_checkpoint_size(self.h, C.byref(nb)), "duwp_checkpoint_size")
        buf = (C.c_ubyte * nb.value)()
        _chk(self.L.duwp_checkpoint_save(self.h, buf, nb.value), "duwp_checkpoint_save")
        return bytes(buf)

    def restore(self, blob: bytes):
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        _chk(self.L.duwp_checkpoint_restore(self.h, buf, len(blob)), "duwp_checkpoint_restore")


class _PartView(Solver):
    """Inspection of one part of a Split (its handle belongs to the split)."""

    def __init__(self, L, h, params: dict, c0: int, c1: int):
        self.L, self.h = L, h
        self.params = [dict(params, n_cells=c1 - c0)]
        self.n = 1
        self.c0, self.c1 = c0, c1

    def close(self):
        self.h = None


class Split:
    """One instance split into `parts` contiguous cell ranges stepped in lockstep (duwp_split_*):
    the exchange of crossing particles and of a one-cell halo every step keeps the results equal to
    the undivided instance's.  devices: one CUDA device per part (default: all on `device`)."""

    def __init__(self, params: dict, parts: int, device: int = 0, devices=None, torch_alloc: bool = True):
        import torch
        L = load()
        if not torch.cuda.is_available():
            raise RuntimeError("the DUWP library needs a CUDA device")
        torch.cuda.set_device(device)
        self.params = params
        self._alloc = _TorchAllocator(device) if (torch_alloc and devices is None) else None
        a = self._alloc.alloc if self._alloc else ALLOC_FN()
        f = self._alloc.free if self._alloc else FREE_FN()
        dv = None
        if devices is not None:
            dv = (C.c_int32 * parts)(*[int(d) for d in devices])
        pr = make_params(params)
        h = C.c_void_p()
        _chk(L.duwp_split_create(C.byref(pr), int(parts), dv, a, f, None, C.byref(h)), "duwp_split_create")
        self.h, self.L = h, L
        self.parts = []
        for r in range(parts):
            ph, c0, c1 = C.c_void_p(), C.c_int32(), C.c_int32()
            _chk(L.duwp_split_part(h, r, C.byref(ph), C.byref(c0), C.byref(c1)), "duwp_split_part")
            self.parts.append(_PartView(L, ph, params, int(c0.value), int(c1.value)))

    def step(self, n: int = 1):
        _chk(self.L.duwp_split_step(self.h, int(n)), "duwp_split_step")

    def fields(self):
        return np.concatenate([p.fields()[0] for p in self.parts])

    def particles(self) -> dict:
        ps = []
        for p in self.parts:
            d = p.particles()
            d["cell"] = d["cell"] + p.c0
            ps.append(d)
        return {k: np.concatenate([d[k] for d in ps]) for k in ps[0]}

    def counters(self) -> dict:
        cs = [p.counters() for p in self.parts]
        return {k: np.concatenate([c[k] for c in cs]) for k in cs[0]}

    def cmax(self) -> np.ndarray:
        return np.concatenate([p.cmax() for p in self.parts])

    def particle_updates(self) -> int:
        return int(sum(p.info(0)["particle_updates"] for p in self.parts))

    def close(self):
        if getattr(self, "h", None):
            for p in self.parts:
                p.close()
            self.L.duwp_split_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (duwp_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, max_cells: int = 0, steps_per_launch: int = 10,
                 precision: str = "fp32", device: int = 0, torch_alloc: bool = True, lanes: int = 1,
                 long_steps: int = 0):
        import torch
        L = load()
        torch.cuda.set_device(device)
        self.stream = torch.cuda.Stream(device=device)
        cfg = ServerCfg(int(hbm_budget_bytes), int(max_slots), int(max_cells), int(steps_per_launch),
                        PRECISION[precision], C.c_void_p(self.stream.cuda_stream), int(lanes), int(long_steps))
        self._alloc = _TorchAllocator(device) if torch_alloc else None
        a = self._alloc.alloc if self._alloc else ALLOC_FN()
        f = self._alloc.free if self._alloc else FREE_FN()
        s = C.c_void_p()
        _chk(L.duwp_server_create(C.byref(cfg), a, f, None, C.byref(s)), "duwp_server_create")
        self.s = s
        self.L = L

    def submit(self, params: dict, n_steps: int) -> int:
        rid = C.c_uint64()
        p = make_params(params)
        _chk(self.L.duwp_submit(self.s, C.byref(p), int(n_steps), C.byref(rid)), "duwp_submit")
        return int(rid.value)

    def poll(self, rid: int):
        """None while pending; a dict once finished (the request is released by this call's
        successor, so the arrays are copied here)."""
        r = Result()
        rc = self.L.duwp_poll(self.s, C.c_uint64(rid), C.byref(r))
        if rc == PENDING:
            return None
        _chk(rc, "duwp_poll")
        n = r.n_cells
        out = {"status": r.status, "n_cells": n, "steps": r.steps, "particle_updates": r.particle_updates,
               "queue_ms": r.queue_ms, "run_ms": r.run_ms, "step_p50_ms": r.step_p50_ms,
               "step_p99_ms": r.step_p99_ms}
        for k in ("rho", "u", "T"):
            ptr = getattr(r, k)
            out[k] = np.ctypeslib.as_array(ptr, shape=(n,)).copy() if (n > 0 and ptr) else np.zeros(0)
        self.L.duwp_poll(self.s, C.c_uint64(rid), C.byref(r))   # release
        return out

    def close(self):
        if getattr(self, "s", None):
            self.L.duwp_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shock_normalised(kind: str, x, rho, T, Pi, Q, up, down, lam_up: float, beta: float = 1.0,
                     R: float = 1.0) -> dict:
    """Shock-structure profiles in the paper's normalisation (Sec. 4.1, Eqs. ma3 / ma8), computed by
    duwp_shock_normalise.  up, down: (rho, T) of the inflow and outflow states; lam_up: the inflow
    mean free path of Eq. (lambda); beta its factor."""
    kinds = {"ma3": 0, "ma8": 1}
    if kind not in kinds:
        raise ValueError(f"unknown normalisation {kind!r} (ma3 | ma8)")
    L = load()
    ins = [np.ascontiguousarray(a, np.float64) for a in (x, rho, T, Pi, Q)]
    n = len(ins[0])
    if any(len(a) != n for a in ins):
        raise ValueError("x, rho, T, Pi and Q must have the same length")
    outs = [np.empty(n, np.float64) for _ in range(5)]
    (r1, T1), (r2, T2) = up, down
    _chk(L.duwp_shock_normalise(kinds[kind], n, *[_dptr(a) for a in ins], float(r1), float(T1), float(r2), float(T2),
                                float(lam_up), float(beta), float(R), *[_dptr(a) for a in outs]),
         "duwp_shock_normalise")
    return dict(zip(("x", "rho", "T", "Pi", "Q"), outs))
