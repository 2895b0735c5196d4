"""Plain FP64 CPU oracle of the DUWP time step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library and its Python binding never import it, and it imports nothing from
them: problems are described by plain dicts (see
``paper_2305_12071_gb300.workloads`` for the seeded generators of those dicts).

The arithmetic lives in ``duwp_oracle.c`` (C99, compiled with
``-ffp-contract=off`` so no multiply-add is fused behind the reader's back);
this module compiles it on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "duwp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC = {"inout": 0, "specular": 1, "periodic": 2, "vacuum": 3}
EPS = {"eps1": 0, "eps12": 1, "eps0": 2, "eps_avg": 3}
FLUX = {"gks_eq": 0, "kfvs": 1}
NTC = {"particle": 0, "total": 1}
RESAMPLE = {"maxwell": 0, "ce": 1}
SPLIT = {"p": 0, "qmc": 1}
RECON = {"first": 0, "vanleer": 1}


class _State(C.Structure):
    _fields_ = [("rho", C.c_double), ("u", C.c_double), ("v", C.c_double), ("w", C.c_double), ("T", C.c_double)]


class _Params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("Pr", C.c_double), ("R", C.c_double),
        ("omega", C.c_double), ("alpha", C.c_double),
        ("rho_ref", C.c_double), ("T_ref", C.c_double), ("Kn", C.c_double), ("L_ref", C.c_double),
        ("x_min", C.c_double), ("x_max", C.c_double),
        ("n_cells", C.c_int32),
        ("dt", C.c_double), ("cfl", C.c_double),
        ("left", _State), ("right", _State),
        ("x_split", C.c_double),
        ("bc_left", C.c_int32), ("bc_right", C.c_int32),
        ("ppc_ref", C.c_double),
        ("fp32", C.c_int32), ("eps_mode", C.c_int32), ("flux_mode", C.c_int32), ("ntc_rate", C.c_int32),
        ("seed", C.c_uint64),
        ("avg_start", C.c_int32),
        ("resample_mode", C.c_int32),
        ("split_mode", C.c_int32),
        ("recon_mode", C.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile duwp_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FP contraction)."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        d, i32, u32, i64, vp = C.c_double, C.c_int32, C.c_uint32, C.c_int64, C.c_void_p
        P = C.POINTER
        L.ora_philox.argtypes = [u32, u32, P(u32), P(u32)]
        L.ora_u53.argtypes = [u32, u32]; L.ora_u53.restype = d
        L.ora_pick_pair.argtypes = [u32, u32, u32, P(u32), P(u32)]
        L.ora_beta.argtypes = [d, d]; L.ora_beta.restype = d
        L.ora_c_ref.argtypes = [d, d, d]; L.ora_c_ref.restype = d
        L.ora_eps.argtypes = [C.c_int, d]; L.ora_eps.restype = d
        L.ora_half_moments.argtypes = [d, d, P(d), P(d)]
        L.ora_wave_flux.argtypes = [P(_Params), P(d), P(d), C.c_int, P(d)]
        L.ora_scatter.argtypes = [d, d, P(d), P(d)]
        L.ora_ntc_nsel.argtypes = [P(_Params), d, d, d]; L.ora_ntc_nsel.restype = d
        L.ora_create.argtypes = [P(_Params)]; L.ora_create.restype = vp
        L.ora_destroy.argtypes = [vp]
        L.ora_step.argtypes = [vp, i32]; L.ora_step.restype = C.c_int
        L.ora_num_particles.argtypes = [vp]; L.ora_num_particles.restype = i64
        L.ora_step_count.argtypes = [vp]; L.ora_step_count.restype = u32
        L.ora_last_nfar.argtypes = [vp]; L.ora_last_nfar.restype = i64
        L.ora_num_last_pre.argtypes = [vp]; L.ora_num_last_pre.restype = i64
        L.ora_get_last_pre.argtypes = [vp, P(i32), P(i64), P(d), P(d), P(d), P(d)]
        L.ora_get_particles.argtypes = [vp, P(i32), P(d), P(d), P(d), P(d)]
        L.ora_set_particles.argtypes = [vp, i64, P(i32), P(d), P(d), P(d), P(d)]
        L.ora_set_particles.restype = C.c_int
        L.ora_get_psi.argtypes = [vp, P(d)]
        L.ora_set_psi.argtypes = [vp, P(d)]
        L.ora_get_avg.argtypes = [vp, P(d)]; L.ora_get_avg.restype = i64
        L.ora_get_cmax.argtypes = [vp, P(d)]
        L.ora_get_last_flux.argtypes = [vp, P(d)]
        L.ora_get_last_moments.argtypes = [vp, P(d), P(d)]
        L.ora_get_counters.argtypes = [vp, P(i32), P(i32), P(i32), P(i32)]
        L.ora_get_consts.argtypes = [vp, P(d)]
        L.ora_get_prim.argtypes = [vp, P(d), P(d), P(d), P(d), P(i32)]
        L.ora_stress_heat.argtypes = [vp, P(d), P(d)]
        L.ora_recon_pair.argtypes = [P(d), P(d), P(d), P(d), P(d), P(d)]
        L.ora_transport.argtypes = [vp, i64, P(d), P(d)]; L.ora_transport.restype = i64
        L.ora_ce_sample.argtypes = [P(_Params), P(d), P(d), P(d), u32, u32, u32, u32, i64, P(d), P(d)]
        L.ora_set_range.argtypes = [vp, i32, i32]; L.ora_set_range.restype = C.c_int
        L.ora_step_first_half.argtypes = [vp]; L.ora_step_first_half.restype = C.c_int
        L.ora_outbox_count.argtypes = [vp]; L.ora_outbox_count.restype = i64
        L.ora_outbox.argtypes = [vp, P(i32), P(d), P(d), P(d), P(d)]
        L.ora_step_second_half.argtypes = [vp, i64, P(i32), P(d), P(d), P(d), P(d),
                                           i64, P(i32), P(d), P(d), P(d), P(d)]
        L.ora_step_second_half.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def make_params(p: dict) -> _Params:
    """Marshal a problem dict (keys as in the workload generators) into the C struct."""
    s = _Params()
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
    s.left = _State(*p["left"])
    s.right = _State(*p["right"])
    s.x_split = p.get("x_split", 0.5 * (p["x_min"] + p["x_max"]))
    s.bc_left = BC[p.get("bc_left", "inout")]
    s.bc_right = BC[p.get("bc_right", "inout")]
    s.ppc_ref = p["ppc_ref"]
    s.fp32 = 1 if p.get("precision", "fp64") == "fp32" else 0
    s.eps_mode = EPS[p.get("eps_mode", "eps1")]
    s.flux_mode = FLUX[p.get("flux_mode", "gks_eq")]
    s.ntc_rate = NTC[p.get("ntc_rate", "particle")]
    s.seed = int(p.get("seed", 1)) & 0xFFFFFFFFFFFFFFFF
    s.avg_start = int(p.get("avg_start", 0))
    s.resample_mode = RESAMPLE[p.get("resample_mode", "maxwell")]
    s.split_mode = SPLIT[p.get("split_mode", "p")]
    s.recon_mode = RECON[p.get("recon_mode", "first")]
    return s


# ---------------------------------------------------------------- pure functions

def philox(key0: int, key1: int, ctr) -> tuple:
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    o = (C.c_uint32 * 4)()
    lib().ora_philox(key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF, c, o)
    return tuple(int(x) for x in o)


def ce_sample(params: dict, Wm, W0, Wp, key=(7, 11), cell_id: int = 1, step: int = 0, n: int = 1000):
    """Chapman-Enskog coefficients (on, sigma_xx, sigma_yy, sigma_xy, sigma_xz, q_x, A) of a cell with
    neighbouring states Wm | W0 | Wp ((rho, u, v, w, T) each) and n velocity samples of that cell."""
    pr = make_params(params)
    arr = lambda x: (C.c_double * 5)(*[float(v) for v in x])
    xi = np.zeros(3 * n, np.float64)
    coef = (C.c_double * 7)()
    lib().ora_ce_sample(C.byref(pr), arr(Wm), arr(W0), arr(Wp), key[0], key[1], cell_id, step, n,
                        xi.ctypes.data_as(C.POINTER(C.c_double)), coef)
    return list(coef), xi.reshape(n, 3)


def recon_pair(Wm, W0, W1, W2):
    """Reconstructed (van Leer) interface states between primitive states W0 and W1."""
    a = [np.ascontiguousarray(x, np.float64) for x in (Wm, W0, W1, W2)]
    L, R = np.empty(5), np.empty(5)
    lib().ora_recon_pair(*[_ptr(x, C.c_double) for x in a], _ptr(L, C.c_double), _ptr(R, C.c_double))
    return L, R


def u53(a: int, b: int) -> float:
    return lib().ora_u53(a & 0xFFFFFFFF, b & 0xFFFFFFFF)


def pick_pair(w0: int, w1: int, n: int) -> tuple:
    a, b = C.c_uint32(), C.c_uint32()
    lib().ora_pick_pair(w0, w1, n, C.byref(a), C.byref(b))
    return a.value, b.value


def beta(omega: float, alpha: float = 1.0) -> float:
    return lib().ora_beta(omega, alpha)


def c_ref(omega: float, R: float = 1.0, T_ref: float = 1.0) -> float:
    return lib().ora_c_ref(omega, R, T_ref)


def eps(mode: str, x: float) -> float:
    return lib().ora_eps(EPS[mode], x)


def half_moments(U: float, lam: float):
    mp, mm = (C.c_double * 4)(), (C.c_double * 4)()
    lib().ora_half_moments(U, lam, mp, mm)
    return np.array(mp[:]), np.array(mm[:])


def wave_flux(params: dict, WL, WR, viscous: bool = True) -> np.ndarray:
    s = make_params(params)
    a = (C.c_double * 5)(*WL)
    b = (C.c_double * 5)(*WR)
    f = (C.c_double * 5)()
    lib().ora_wave_flux(C.byref(s), a, b, 1 if viscous else 0, f)
    return np.array(f[:])


def scatter(r1: float, r2: float, a, b):
    A = (C.c_double * 3)(*a)
    B = (C.c_double * 3)(*b)
    lib().ora_scatter(r1, r2, A, B)
    return np.array(A[:]), np.array(B[:])


def ntc_nsel(params: dict, rho_ratio: float, n: float, cmax: float) -> float:
    s = make_params(params)
    return lib().ora_ntc_nsel(C.byref(s), rho_ratio, n, cmax)


# ---------------------------------------------------------------- instance

class Oracle:
    """One DUWP instance stepped by the plain C oracle."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self._p = make_params(params)
        self.h = lib().ora_create(C.byref(self._p))
        if not self.h:
            raise ValueError("oracle rejected the problem description")
        self.C = int(params["n_cells"])

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().ora_destroy(h)
            self.h = None

    def step(self, n: int = 1):
        rc = lib().ora_step(self.h, int(n))
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")

    @property
    def steps_done(self) -> int:
        return int(lib().ora_step_count(self.h))

    def psi(self) -> np.ndarray:
        out = np.empty((self.C, 5), np.float64)
        lib().ora_get_psi(self.h, _ptr(out, C.c_double))
        return out

    def set_psi(self, psi: np.ndarray):
        a = np.ascontiguousarray(psi, np.float64)
        lib().ora_set_psi(self.h, _ptr(a, C.c_double))

    def avg(self):
        out = np.empty((self.C, 5), np.float64)
        n = lib().ora_get_avg(self.h, _ptr(out, C.c_double))
        return out, int(n)

    def cmax(self) -> np.ndarray:
        out = np.empty(self.C, np.float64)
        lib().ora_get_cmax(self.h, _ptr(out, C.c_double))
        return out

    def last_flux(self) -> np.ndarray:
        out = np.empty((self.C + 1, 5), np.float64)
        lib().ora_get_last_flux(self.h, _ptr(out, C.c_double))
        return out

    def last_moments(self):
        pre = np.empty((self.C, 5), np.float64)
        post = np.empty((self.C, 5), np.float64)
        lib().ora_get_last_moments(self.h, _ptr(pre, C.c_double), _ptr(post, C.c_double))
        return pre, post

    def num_particles(self) -> int:
        return int(lib().ora_num_particles(self.h))

    def last_nfar(self) -> int:
        return int(lib().ora_last_nfar(self.h))

    def particles(self) -> dict:
        n = self.num_particles()
        cell = np.empty(n, np.int32)
        xl, u, v, w = (np.empty(n, np.float64) for _ in range(4))
        lib().ora_get_particles(self.h, _ptr(cell, C.c_int32), _ptr(xl, C.c_double), _ptr(u, C.c_double),
                                _ptr(v, C.c_double), _ptr(w, C.c_double))
        return {"cell": cell, "xl": xl, "u": u, "v": v, "w": w}

    def last_pre(self) -> dict:
        n = int(lib().ora_num_last_pre(self.h))
        src = np.empty(n, np.int32)
        dest = np.empty(n, np.int64)
        xl, u, v, w = (np.empty(n, np.float64) for _ in range(4))
        lib().ora_get_last_pre(self.h, _ptr(src, C.c_int32), _ptr(dest, C.c_int64), _ptr(xl, C.c_double),
                               _ptr(u, C.c_double), _ptr(v, C.c_double), _ptr(w, C.c_double))
        return {"src": src, "dest": dest, "xl": xl, "u": u, "v": v, "w": w}

    def set_particles(self, cell, xl, u, v, w):
        cell = np.ascontiguousarray(cell, np.int32)
        arrs = [np.ascontiguousarray(a, np.float64) for a in (xl, u, v, w)]
        rc = lib().ora_set_particles(self.h, len(cell), _ptr(cell, C.c_int32),
                                     *[_ptr(a, C.c_double) for a in arrs])
        if rc != 0:
            raise ValueError("particles must be sorted by cell and inside the domain")

    def counters(self) -> dict:
        out = {k: np.empty(self.C, np.int32) for k in ("ncand", "nacc", "nabs", "nnew")}
        lib().ora_get_counters(self.h, *[_ptr(out[k], C.c_int32) for k in ("ncand", "nacc", "nabs", "nnew")])
        return out

    def consts(self) -> dict:
        o = (C.c_double * 10)()
        lib().ora_get_consts(self.h, o)
        keys = ("dx", "dt", "dtdx", "mp", "beta", "lambda_ref", "mu_ref", "upsilon", "c_ref", "ntc_A")
        return dict(zip(keys, o[:]))

    def prim(self) -> dict:
        rho, u, T, P = (np.empty(self.C, np.float64) for _ in range(4))
        valid = np.empty(self.C, np.int32)
        lib().ora_get_prim(self.h, _ptr(rho, C.c_double), _ptr(u, C.c_double), _ptr(T, C.c_double),
                           _ptr(P, C.c_double), _ptr(valid, C.c_int32))
        return {"rho": rho, "u": u, "T": T, "P": P, "valid": valid.astype(bool)}

    def stress_heat(self) -> dict:
        """Normal stress Pi = S_xx and heat flux Q = Q_x per cell (Eq. gkt_moment1) of the current
        state: particle central moments about U_t plus the wave's NS values weighted by rho_w/rho_t."""
        Pi, Q = np.empty(self.C, np.float64), np.empty(self.C, np.float64)
        lib().ora_stress_heat(self.h, _ptr(Pi, C.c_double), _ptr(Q, C.c_double))
        return {"Pi": Pi, "Q": Q}

    # ---------------------------------------------------------------- domain decomposition
    def set_range(self, c0: int, c1: int):
        """Own only cells [c0, c1) (one part of a domain split; before the first step)."""
        if lib().ora_set_range(self.h, int(c0), int(c1)) != 0:
            raise ValueError("bad cell range")
        self.c0, self.c1 = int(c0), int(c1)

    def first_half(self):
        """Step 1, Step 2 of the owned cells and the transport (Step 3) of their particles."""
        if lib().ora_step_first_half(self.h) != 0:
            raise RuntimeError("first half failed")

    def outbox(self) -> dict:
        """Transported particles whose new cell another part owns, in pre-transport order."""
        n = int(lib().ora_outbox_count(self.h))
        if n < 0:
            raise RuntimeError("no first half taken")
        cell = np.empty(n, np.int32)
        xl, u, v, w = (np.empty(n, np.float64) for _ in range(4))
        lib().ora_outbox(self.h, _ptr(cell, C.c_int32), _ptr(xl, C.c_double), _ptr(u, C.c_double),
                         _ptr(v, C.c_double), _ptr(w, C.c_double))
        return {"cell": cell, "xl": xl, "u": u, "v": v, "w": w}

    def second_half(self, lo: dict, hi: dict):
        """New particle lists of the owned cells from this part's transported particles and those
        arriving from lower (lo) and higher (hi) parts, then the update of the owned cells."""
        def args(d):
            c = np.ascontiguousarray(d["cell"], np.int32)
            a = [np.ascontiguousarray(d[k], np.float64) for k in ("xl", "u", "v", "w")]
            return [len(c), _ptr(c, C.c_int32)] + [_ptr(x, C.c_double) for x in a], (c, a)
        la, keep_lo = args(lo)
        ha, keep_hi = args(hi)
        if lib().ora_step_second_half(self.h, *la, *ha) != 0:
            raise RuntimeError("second half failed (an arriving particle outside the owned range?)")

    def transport(self, cell: int, xl: float, u: float):
        x, uu = C.c_double(xl), C.c_double(u)
        d = lib().ora_transport(self.h, cell, C.byref(x), C.byref(uu))
        return int(d), x.value, uu.value


# ---------------------------------------------------------------------------- domain decomposition
def split_ranges(n_cells: int, parts: int):
    """Contiguous cell ranges [c0, c1) of `parts` parts of nearly equal size."""
    edges = [(n_cells * r) // parts for r in range(parts + 1)]
    return [(edges[r], edges[r + 1]) for r in range(parts)]


def halo_cells(n_cells: int, c0: int, c1: int, periodic: bool, width: int = 2):
    """Cells outside [c0, c1) whose states the owned cells read: `width` on each side (the wave flux
    with the second-order reconstruction reads two; the flux and the NS-corrected sampling one),
    wrapping at periodic ends."""
    out = []
    for k in range(1, width + 1):
        for c in (c0 - k, c1 - 1 + k):
            if periodic:
                c %= n_cells
            if 0 <= c < n_cells and not (c0 <= c < c1) and c not in out:
                out.append(c)
    return out


def route(outboxes, ranges, me: int):
    """Particles arriving in part `me` from every part's outbox (outboxes[r], pre-transport order):
    (from lower parts, from higher parts), each concatenated in part order."""
    c0, c1 = ranges[me]
    lo, hi = [], []
    for r, box in enumerate(outboxes):
        if r == me:
            continue
        sel = (box["cell"] >= c0) & (box["cell"] < c1)
        piece = {k: v[sel] for k, v in box.items()}
        (lo if r < me else hi).append(piece)

    def cat(pieces):
        if not pieces:
            return {"cell": np.empty(0, np.int32), **{k: np.empty(0) for k in ("xl", "u", "v", "w")}}
        return {k: np.concatenate([p[k] for p in pieces]) for k in pieces[0]}
    return cat(lo), cat(hi)


class DomainSplit:
    """One instance split into `parts` contiguous cell ranges, each held by its own oracle instance
    that owns only its cells: the host-rank emulation of a one-instance multi-GPU run.  Every step
    exchanges the states of the cells next to each range (halo) before the first half and the
    particles that cross into another range between the halves."""

    def __init__(self, params: dict, parts: int):
        self.C = int(params["n_cells"])
        self.periodic = params.get("bc_left") == "periodic"
        self.ranges = split_ranges(self.C, parts)
        self.parts = []
        for c0, c1 in self.ranges:
            o = Oracle(params)
            o.set_range(c0, c1)
            self.parts.append(o)

    def psi(self) -> np.ndarray:
        full = np.zeros((self.C, 5))
        for o, (c0, c1) in zip(self.parts, self.ranges):
            full[c0:c1] = o.psi()[c0:c1]
        return full

    def step(self, n: int = 1):
        for _ in range(n):
            full = self.psi()
            for o, (c0, c1) in zip(self.parts, self.ranges):
                mine = o.psi()
                view = np.zeros_like(mine)
                view[c0:c1] = mine[c0:c1]
                for c in halo_cells(self.C, c0, c1, self.periodic):
                    view[c] = full[c]
                o.set_psi(view)
                o.first_half()
            boxes = [o.outbox() for o in self.parts]
            for me, o in enumerate(self.parts):
                lo, hi = route(boxes, self.ranges, me)
                o.second_half(lo, hi)

    def particles(self) -> dict:
        ps = [o.particles() for o in self.parts]
        return {k: np.concatenate([p[k] for p in ps]) for k in ps[0]}

    def counters(self) -> dict:
        out = {k: np.zeros(self.C, np.int32) for k in ("ncand", "nacc", "nabs", "nnew")}
        for o, (c0, c1) in zip(self.parts, self.ranges):
            c = o.counters()
            for k in out:
                out[k][c0:c1] = c[k][c0:c1]
        return out

    def cmax(self) -> np.ndarray:
        out = np.zeros(self.C)
        for o, (c0, c1) in zip(self.parts, self.ranges):
            out[c0:c1] = o.cmax()[c0:c1]
        return out

