"""CPU oracle for the FF-SRL batched XPBD step (arXiv 2503.18616).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers allowed. The simulator
package never imports this module and shares no code with it.

The arithmetic lives in ``xpbd_oracle.c`` (plain sequential C, FP64). This file
only compiles it with gcc and marshals numpy arrays through ctypes. A second
build with ``REAL=float`` ("f32") exists to measure the FP32 rounding floor.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .mlp import *  # noqa: F401,F403  (FP64 network oracle, pure numpy)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xpbd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[str, ctypes.CDLL] = {}


def lib_path(precision: str = "f64") -> str:
    return os.path.join(_BUILD, f"liboracle_{precision}.so")


def build(precision: str = "f64", force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so the C reads as run)."""
    out = lib_path(precision)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    real = "double" if precision == "f64" else "float"
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           f"-DREAL={real}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(precision: str = "f64") -> ctypes.CDLL:
    with _LOCK:
        if precision not in _LIBS:
            L = ctypes.CDLL(build(precision))
            P, I, D, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
            L.orc_mix64.restype = U64
            L.orc_mix64.argtypes = [U64]
            L.orc_sm64.restype = U64
            L.orc_sm64.argtypes = [U64, U64]
            L.orc_stream.restype = U64
            L.orc_stream.argtypes = [U64, U64, ctypes.c_uint32]
            L.orc_uniform_pm1.restype = D
            L.orc_uniform_pm1.argtypes = [U64]
            L.orc_action.restype = D
            L.orc_action.argtypes = [U64, U64, U64, I]
            L.orc_sample_indices.restype = I
            L.orc_sample_indices.argtypes = [U64, U64, I, I, P]
            L.orc_target_index.restype = I
            L.orc_target_index.argtypes = [U64, U64, I]
            L.orc_env_set_clamp.argtypes = [P, D]
            L.orc_env_grasper.argtypes = [P, P, P, P, P]
            L.orc_episode_seed.restype = U64
            L.orc_episode_seed.argtypes = [U64, I]
            L.orc_mesh_create.restype = P
            L.orc_mesh_create.argtypes = [I, P, P, I, P, I, P, D, ctypes.POINTER(I)]
            L.orc_mesh_destroy.argtypes = [P]
            L.orc_mesh_info.argtypes = [P, P]
            L.orc_mesh_faces.argtypes = [P, P]
            L.orc_closest_segment_triangle.restype = D
            L.orc_closest_segment_triangle.argtypes = [P, P, P, P, P, P, P, P]
            L.orc_mesh_get_int.argtypes = [P, I, P]
            L.orc_mesh_get_real.argtypes = [P, I, P]
            L.orc_env_create.restype = P
            L.orc_env_create.argtypes = [P]
            L.orc_env_destroy.argtypes = [P]
            L.orc_env_reset.restype = I
            L.orc_env_reset.argtypes = [P, P, U64, U64]
            L.orc_env_step.restype = I
            L.orc_env_step.argtypes = [P, P, P, D, P, P, P]
            L.orc_env_run.restype = I
            L.orc_env_run.argtypes = [P, P, I, P, D, P, P, P]
            L.orc_env_get.argtypes = [P, P, P, P]
            L.orc_env_set.argtypes = [P, P, P, P]
            L.orc_env_get_ints.argtypes = [P, P]
            L.orc_env_get_tool_box.argtypes = [P, P, P]
            L.orc_obs_dim.restype = I
            L.orc_obs_dim.argtypes = [P]
            L.orc_real_size.restype = I
            R = D if precision == "f64" else ctypes.c_float
            L.orc_project_edge.restype = R
            L.orc_project_edge.argtypes = [P, P, R, R, R, R, P, R]
            L.orc_mesh_conns.argtypes = [P, P]
            L.orc_project_conn.restype = R
            L.orc_project_conn.argtypes = [P, P, P, P, P, R, R, P, R]
            L.orc_project_tet.restype = R
            L.orc_project_tet.argtypes = [P, P, P, P, P, R, R, P]
            L.orc_mlp_forward.argtypes = [P, P, P]
            L.orc_env_residual.restype = D
            L.orc_env_residual.argtypes = [P]
            L.orc_env_features.argtypes = [P, P, P]
            L.orc_env_step_surrogate.restype = I
            L.orc_env_step_surrogate.argtypes = [P, P, P, D, P, D, I, P, P, P, P, P, P, P]
            _LIBS[precision] = L
        return _LIBS[precision]


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------
# Random numbers (SplitMix64, counter-based)
# --------------------------------------------------------------------------

def mix64(z: int) -> int:
    return int(_lib().orc_mix64(z & (2**64 - 1)))


def sm64(state: int, n: int) -> int:
    return int(_lib().orc_sm64(state & (2**64 - 1), n))


def stream(seed: int, env: int, domain: int) -> int:
    return int(_lib().orc_stream(seed, env, domain))


def uniform_pm1(r: int) -> float:
    return float(_lib().orc_uniform_pm1(r))


def action(seed: int, env: int, t: int, axis: int) -> float:
    return float(_lib().orc_action(seed, env, t, axis))


def sample_indices(seed: int, env: int, n: int, k: int) -> np.ndarray:
    out = np.zeros(max(k, 1), dtype=np.int32)
    rc = _lib().orc_sample_indices(seed, env, n, k, _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_sample_indices rc={rc}")
    return out[:k].copy()


def episode_seed(seed0: int, k: int) -> int:
    """Seed of episode k >= 1 started by auto-reset."""
    return int(_lib().orc_episode_seed(seed0, k))


def target_index(seed: int, env: int, n: int) -> int:
    return int(_lib().orc_target_index(seed, env, n))


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------

class Params(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double),
        ("substeps", ctypes.c_int),
        ("iterations", ctypes.c_int),
        ("gravity", ctypes.c_double * 3),
        ("alpha_d", ctypes.c_double),
        ("alpha_v", ctypes.c_double),
        ("radius", ctypes.c_double),
        ("action_scale", ctypes.c_double),
        ("margin_xy", ctypes.c_double),
        ("margin_below", ctypes.c_double),
        ("margin_above", ctypes.c_double),
        ("w_l", ctypes.c_double),
        ("w_d", ctypes.c_double),
        ("w_s", ctypes.c_double),
        ("success_dist", ctypes.c_double),
        ("n_obs", ctypes.c_int),
        ("max_steps", ctypes.c_int),
        ("solver", ctypes.c_int),
        ("auto_reset", ctypes.c_int),
        ("tool_model", ctypes.c_int),
        ("rcm_height", ctypes.c_double),
        ("shaft_radius", ctypes.c_double),
        ("clamp_length", ctypes.c_double),
        ("clamp_radius", ctypes.c_double),
        ("clamp_angle", ctypes.c_double),
        ("grasp_radius", ctypes.c_double),
    ]

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        p = cls()
        for name, _ in cls._fields_:
            val = d.get(name, 0) if name in ("solver", "auto_reset", "tool_model", "rcm_height", "shaft_radius",
                                             "clamp_length", "clamp_radius", "clamp_angle", "grasp_radius") else d[name]
            if name == "gravity":
                p.gravity[:] = [float(g) for g in val]
            else:
                setattr(p, name, val)
        return p


class Net(ctypes.Structure):
    """Warm-start network parameters with frozen normalisation (orc_mlp)."""
    _fields_ = [
        ("W1", (ctypes.c_double * 15) * 64), ("b1", ctypes.c_double * 64),
        ("W2", (ctypes.c_double * 64) * 64), ("b2", ctypes.c_double * 64),
        ("W3", (ctypes.c_double * 64) * 3), ("b3", ctypes.c_double * 3),
        ("in_mean", ctypes.c_double * 15), ("in_std", ctypes.c_double * 15),
        ("out_mean", ctypes.c_double * 3), ("out_std", ctypes.c_double * 3),
        ("bf16", ctypes.c_int),
    ]

    @classmethod
    def from_params(cls, p: dict, in_mean=None, in_std=None, out_mean=None, out_std=None, bf16=False):
        n = cls()
        for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
            arr = np.ascontiguousarray(p[k], dtype=np.float64)
            ctypes.memmove(ctypes.addressof(getattr(n, k)), arr.ctypes.data, arr.nbytes)
        for k, val, size in (("in_mean", in_mean, 15), ("in_std", in_std, 15),
                             ("out_mean", out_mean, 3), ("out_std", out_std, 3)):
            default = 0.0 if "mean" in k else 1.0
            arr = np.full(size, default) if val is None else np.ascontiguousarray(val, dtype=np.float64)
            ctypes.memmove(ctypes.addressof(getattr(n, k)), arr.ctypes.data, arr.nbytes)
        n.bf16 = int(bool(bf16))
        return n


def net_forward(net: "Net", feats) -> np.ndarray:
    """The C oracle's network on feature rows [n][15] (de-normalised output [n][3])."""
    L = _lib()
    F = np.ascontiguousarray(feats, dtype=np.float64).reshape(-1, 15)
    out = np.zeros((len(F), 3))
    for i in range(len(F)):
        L.orc_mlp_forward(ctypes.byref(net), _ptr(F[i]), _ptr(out[i]))
    return out


# --------------------------------------------------------------------------
# Mesh and environment
# --------------------------------------------------------------------------

class Mesh:
    """Constraint tables built by the oracle from a tet mesh."""

    def __init__(self, rest, inv_mass, tets, edges=None, precision: str = "f64", conn_radius: float = 0.0):
        self.precision = precision
        self._L = _lib(precision)
        rest = np.ascontiguousarray(rest, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(inv_mass, dtype=np.float64).reshape(-1)
        tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        err = ctypes.c_int(0)
        if edges is not None:
            edges = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
            h = self._L.orc_mesh_create(len(rest), _ptr(rest), _ptr(w), len(tets), _ptr(tets),
                                        len(edges), _ptr(edges), float(conn_radius), ctypes.byref(err))
        else:
            h = self._L.orc_mesh_create(len(rest), _ptr(rest), _ptr(w), len(tets), _ptr(tets),
                                        0, None, float(conn_radius), ctypes.byref(err))
        if not h:
            raise ValueError(f"oracle mesh rejected (code {err.value})")
        self._h = ctypes.c_void_p(h)
        self.error = err.value
        info = np.zeros(6, dtype=np.int32)
        self._L.orc_mesh_info(self._h, _ptr(info))
        self.V, self.T, self.E, self.n_ecol, self.n_tcol, self.n_top = (int(v) for v in info)
        fi = np.zeros(2, dtype=np.int32)
        self._L.orc_mesh_faces(self._h, _ptr(fi))
        self.F, self.n_fcol = int(fi[0]), int(fi[1])
        ci = np.zeros(3, dtype=np.int32)
        self._L.orc_mesh_conns(self._h, _ptr(ci))
        self.C, self.n_ccol, self.n_obj = int(ci[0]), int(ci[1]), int(ci[2])
        self.rest = rest.copy()
        self.inv_mass = w.copy()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_mesh_destroy(h)
            self._h = None

    def _ints(self, which: int, n: int) -> np.ndarray:
        out = np.zeros(max(n, 1), dtype=np.int32)
        self._L.orc_mesh_get_int(self._h, which, _ptr(out))
        return out[:n].copy()

    def _reals(self, which: int, n: int) -> np.ndarray:
        out = np.zeros(max(n, 1), dtype=np.float64)
        self._L.orc_mesh_get_real(self._h, which, _ptr(out))
        return out[:n].copy()

    @property
    def tets(self): return self._ints(0, 4 * self.T).reshape(-1, 4)
    @property
    def flipped(self): return self._ints(1, self.T)
    @property
    def edges(self): return self._ints(2, 2 * self.E).reshape(-1, 2)
    @property
    def ecolor(self): return self._ints(3, self.E)
    @property
    def tcolor(self): return self._ints(4, self.T)
    @property
    def eorder(self): return self._ints(5, self.E)
    @property
    def torder(self): return self._ints(6, self.T)
    @property
    def ecol_off(self): return self._ints(7, self.n_ecol + 1)
    @property
    def tcol_off(self): return self._ints(8, self.n_tcol + 1)
    @property
    def top(self): return self._ints(9, self.n_top)
    @property
    def faces(self): return self._ints(10, 3 * self.F).reshape(-1, 3)
    @property
    def face_opposite(self): return self._ints(11, self.F)
    @property
    def forder(self): return self._ints(12, self.F)
    @property
    def fcol_off(self): return self._ints(13, self.n_fcol + 1)
    @property
    def conns(self): return self._ints(14, 4 * self.C).reshape(-1, 4)
    @property
    def corder(self): return self._ints(15, self.C)
    @property
    def ccol_off(self): return self._ints(16, self.n_ccol + 1)
    @property
    def objects(self): return self._ints(17, self.V)
    @property
    def conn_d0(self): return self._reals(5, self.C)
    @property
    def rest_len(self): return self._reals(0, self.E)
    @property
    def V0(self): return self._reals(1, self.T)
    @property
    def bbmin(self): return self._reals(2, 3)
    @property
    def bbmax(self): return self._reals(3, 3)
    @property
    def extent(self): return float(self._reals(4, 1)[0])


class Env:
    """One environment advanced by the oracle, one step at a time."""

    def __init__(self, mesh: Mesh, params: dict):
        self.mesh = mesh
        self._L = mesh._L
        self.params = dict(params)
        self._p = Params.from_dict(self.params)
        self._h = ctypes.c_void_p(self._L.orc_env_create(mesh._h))
        self.obs_dim = int(self._L.orc_obs_dim(ctypes.byref(self._p)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_env_destroy(h)
            self._h = None

    def reset(self, seed: int, env: int = 0) -> None:
        rc = self._L.orc_env_reset(self._h, ctypes.byref(self._p), seed, env)
        if rc != 0:
            raise ValueError(f"orc_env_reset rc={rc}")

    def step(self, action=None, alpha_d: float = -1.0):
        obs = np.zeros(self.obs_dim, dtype=np.float64)
        rew = np.zeros(1, dtype=np.float64)
        done = np.zeros(1, dtype=np.uint8)
        a = None
        if action is not None:
            a = np.ascontiguousarray(action, dtype=np.float64).reshape(3)
        rc = self._L.orc_env_step(self._h, ctypes.byref(self._p), _ptr(a) if a is not None else None,
                                  float(alpha_d), _ptr(obs), _ptr(rew), _ptr(done))
        if rc != 0:
            raise ValueError(f"orc_env_step rc={rc}")
        return obs, float(rew[0]), int(done[0])

    def run(self, n: int, actions=None, alpha_d: float = -1.0, want_obs: bool = True):
        obs = np.zeros((n, self.obs_dim), dtype=np.float64) if want_obs else None
        rew = np.zeros(n, dtype=np.float64)
        done = np.zeros(n, dtype=np.uint8)
        a = None
        if actions is not None:
            a = np.ascontiguousarray(actions, dtype=np.float64).reshape(n, 3)
        rc = self._L.orc_env_run(self._h, ctypes.byref(self._p), n,
                                 _ptr(a) if a is not None else None, float(alpha_d),
                                 _ptr(obs) if obs is not None else None, _ptr(rew), _ptr(done))
        if rc != 0:
            raise ValueError(f"orc_env_run rc={rc}")
        return obs, rew, done

    def state(self):
        x = np.zeros((self.mesh.V, 3)); v = np.zeros((self.mesh.V, 3)); c = np.zeros(3)
        self._L.orc_env_get(self._h, _ptr(x), _ptr(v), _ptr(c))
        return x, v, c

    def set_state(self, x=None, v=None, c=None):
        args = []
        keep = []
        for a, shape in ((x, (self.mesh.V, 3)), (v, (self.mesh.V, 3)), (c, (3,))):
            if a is None:
                args.append(None)
            else:
                arr = np.ascontiguousarray(a, dtype=np.float64).reshape(shape)
                keep.append(arr)
                args.append(_ptr(arr))
        self._L.orc_env_set(self._h, *args)

    def ints(self):
        out = np.zeros(4 + 2 * self.mesh.V + 8, dtype=np.int32)
        self._L.orc_env_get_ints(self._h, _ptr(out))
        t, target, n_obs, n_c = (int(v) for v in out[:4])
        obs_ids = out[4:4 + n_obs].copy()
        contacts = out[4 + n_obs:4 + n_obs + n_c].copy()
        return {"t": t, "target": target, "obs_ids": obs_ids, "contacts": contacts,
                "episode": int(out[4 + n_obs + n_c]), "grasp": int(out[5 + n_obs + n_c])}

    def grasper(self):
        """The grasper at the current tool point: capsule segments [3][2][3]
        (shaft, clamp +, clamp -), radii [3] and the dragging point [3]."""
        seg, rad, drag = np.zeros((3, 2, 3)), np.zeros(3), np.zeros(3)
        self._L.orc_env_grasper(self._h, ctypes.byref(self._p), _ptr(seg), _ptr(rad), _ptr(drag))
        return seg, rad, drag

    def set_clamp(self, angle: float) -> None:
        """Grasper clamp opening (radians) from the next step on."""
        self._L.orc_env_set_clamp(self._h, float(angle))

    def features(self) -> np.ndarray:
        """Features [V][15] of the next substep's predicted state."""
        F = np.zeros((self.mesh.V, 15))
        self._L.orc_env_features(self._h, ctypes.byref(self._p), _ptr(F))
        return F

    def residual(self) -> float:
        return float(self._L.orc_env_residual(self._h))

    def step_surrogate(self, net, threshold: float, n_full: int, action=None, alpha_d: float = -1.0,
                       residuals=None):
        """Surrogate-assisted step; returns (obs, reward, done, fallbacks).
        `residuals` (a float64 array [substeps], optional) receives the
        residual each substep checked against the threshold."""
        obs = np.zeros(self.obs_dim)
        rew = np.zeros(1)
        done = np.zeros(1, dtype=np.uint8)
        fb = np.zeros(1, dtype=np.int32)
        a = None if action is None else np.ascontiguousarray(action, dtype=np.float64).reshape(3)
        if residuals is not None:
            assert residuals.dtype == np.float64 and residuals.size >= self.params["substeps"]
        rc = self._L.orc_env_step_surrogate(self._h, ctypes.byref(self._p), _ptr(a) if a is not None else None,
                                            float(alpha_d), ctypes.byref(net), float(threshold), int(n_full),
                                            _ptr(obs), _ptr(rew), _ptr(done), _ptr(fb), None, None,
                                            _ptr(residuals) if residuals is not None else None)
        if rc != 0:
            raise ValueError(f"orc_env_step_surrogate rc={rc}")
        return obs, float(rew[0]), int(done[0]), int(fb[0])

    def step_record(self, n_full: int, action=None, alpha_d: float = -1.0):
        """Plain step with `n_full` iterations recording per substep the
        features [S][V][15] and targets [S][V][3] (solve minus prediction)."""
        S, V = self.params["substeps"], self.mesh.V
        F = np.zeros((S, V, 15))
        T = np.zeros((S, V, 3))
        a = None if action is None else np.ascontiguousarray(action, dtype=np.float64).reshape(3)
        rc = self._L.orc_env_step_surrogate(self._h, ctypes.byref(self._p), _ptr(a) if a is not None else None,
                                            float(alpha_d), None, 0.0, int(n_full), None, None, None, None,
                                            _ptr(F), _ptr(T), None)
        if rc != 0:
            raise ValueError(f"orc_env_step_surrogate rc={rc}")
        return F, T

    def tool_box(self):
        lo = np.zeros(3); hi = np.zeros(3)
        self._L.orc_env_get_tool_box(self._h, _ptr(lo), _ptr(hi))
        return lo, hi


# --------------------------------------------------------------------------
# Single-constraint projections (exposed for the pins)
# --------------------------------------------------------------------------

def closest_segment_triangle(q0, q1, a, b, c, precision="f64"):
    """(distance, point on triangle, point on segment, barycentric weights)."""
    dt = np.float64 if precision == "f64" else np.float32
    args = [np.ascontiguousarray(v, dtype=dt) for v in (q0, q1, a, b, c)]
    p, q, w = np.zeros(3, dt), np.zeros(3, dt), np.zeros(3, dt)
    d = _lib(precision).orc_closest_segment_triangle(*[_ptr(v) for v in args], _ptr(p), _ptr(q), _ptr(w))
    return float(d), p, q, w


def project_edge(xa, xb, wa, wb, d, alpha_t, lam=0.0, min_len=0.0, precision="f64"):
    dt = np.float64 if precision == "f64" else np.float32
    a = np.array(xa, dtype=dt); b = np.array(xb, dtype=dt); L = np.array([lam], dtype=dt)
    C = _lib(precision).orc_project_edge(_ptr(a), _ptr(b), wa, wb, d, alpha_t, _ptr(L), min_len)
    return a, b, float(L[0]), float(C)


def project_tet(x4, w4, V0, alpha_t, lam=0.0, precision="f64"):
    dt = np.float64 if precision == "f64" else np.float32
    xs = [np.array(x, dtype=dt) for x in x4]
    w = np.array(w4, dtype=dt); L = np.array([lam], dtype=dt)
    C = _lib(precision).orc_project_tet(_ptr(xs[0]), _ptr(xs[1]), _ptr(xs[2]), _ptr(xs[3]), _ptr(w),
                                        V0, alpha_t, _ptr(L))
    return xs, float(L[0]), float(C)


def project_conn(x4, w4, d0, alpha_t, lam=0.0, min_len=0.0, precision="f64"):
    """Tissue connection (R16) of vertex x4[0] to the centroid of x4[1..3]."""
    dt = np.float64 if precision == "f64" else np.float32
    xs = [np.array(x, dtype=dt) for x in x4]
    w = np.array(w4, dtype=dt); L = np.array([lam], dtype=dt)
    C = _lib(precision).orc_project_conn(_ptr(xs[0]), _ptr(xs[1]), _ptr(xs[2]), _ptr(xs[3]), _ptr(w),
                                         d0, alpha_t, _ptr(L), min_len)
    return xs, float(L[0]), float(C)
