"""Thin Python binding of libffsrl.so (include/ffsrl.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels. PyTorch provides device memory (the tensors whose data pointers
are passed through the C ABI) and the CUDA stream. There is no fallback: if the
compiled library is missing this module raises instead of computing anything.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffsrl.so")
_lib = None

FFSRL_OK = 0
ERRORS = {-1: "FFSRL_E_INVAL", -2: "FFSRL_E_CUDA", -3: "FFSRL_E_OOM", -4: "FFSRL_E_DEGENERATE",
          -5: "FFSRL_E_NAN", -6: "FFSRL_E_TIMEOUT"}

# ffsrl_get_mesh_table selectors
TABLES = {"tets": 0, "flipped": 1, "edges": 2, "ecolor": 3, "tcolor": 4, "eorder": 5,
          "torder": 6, "ecol_off": 7, "tcol_off": 8, "top": 9, "faces": 10, "face_opposite": 11,
          "forder": 12, "fcol_off": 13, "conns": 14, "corder": 15, "ccol_off": 16, "objects": 17}

# every symbol include/ffsrl.h and include/ffsrl_probe.h declare
EXPORTS = ["ffsrl_create", "ffsrl_reset", "ffsrl_step", "ffsrl_step_host", "ffsrl_sync",
           "ffsrl_destroy", "ffsrl_get_info", "ffsrl_last_error", "ffsrl_get_state",
           "ffsrl_set_state", "ffsrl_get_mesh_table", "ffsrl_get_env_ints", "ffsrl_step_noalloc",
           "ffsrl_set_network", "ffsrl_network_forward", "ffsrl_step_surrogate", "ffsrl_record_step",
           "ffsrl_get_rows", "ffsrl_get_network", "ffsrl_network_gradient", "ffsrl_train_network",
           "ffsrl_set_surrogate_envs", "ffsrl_set_clamp_angles", "ffsrl_get_grasp", "ffsrl_network_adam_step",
           "ffsrl_network_normalisation", "ffsrl_probe_fp32", "ffsrl_probe_smem", "ffsrl_set_env_ids"]

NOALLOC_SCRATCH_BYTES = 32 << 20
NET_PARAMS = 64 * 15 + 64 + 64 * 64 + 64 + 3 * 64 + 3   # FFSRL_NET_PARAMS
NET_NORM = 15 + 15 + 3 + 3                              # FFSRL_NET_NORM


class FfsrlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class ffsrl_mesh(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int32), ("n_tets", ctypes.c_int32),
                ("rest_pos", ctypes.c_void_p), ("inv_mass", ctypes.c_void_p),
                ("tets", ctypes.c_void_p)]


class ffsrl_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("substeps", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("gravity", ctypes.c_double * 3), ("compliance_dist", ctypes.c_double),
                ("compliance_vol", ctypes.c_double), ("tool_radius", ctypes.c_double),
                ("action_scale", ctypes.c_double), ("tool_margin_xy", ctypes.c_double),
                ("tool_margin_below", ctypes.c_double), ("tool_margin_above", ctypes.c_double),
                ("w_l", ctypes.c_double), ("w_d", ctypes.c_double), ("w_s", ctypes.c_double),
                ("success_dist", ctypes.c_double), ("n_obs_verts", ctypes.c_int32),
                ("max_steps", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("schedule_flags", ctypes.c_int32), ("solver", ctypes.c_int32), ("auto_reset", ctypes.c_int32),
                ("tool_model", ctypes.c_int32), ("reserved", ctypes.c_int32), ("rcm_height", ctypes.c_double),
                ("shaft_radius", ctypes.c_double), ("clamp_length", ctypes.c_double),
                ("clamp_radius", ctypes.c_double), ("clamp_angle", ctypes.c_double),
                ("grasp_radius", ctypes.c_double), ("conn_radius", ctypes.c_double)]

SCHED_FORCE, SCHED_NO_PERMUTE, SCHED_NO_RING, SCHED_ENVS2, SCHED_ENVS4 = 1, 2, 4, 8, 16
SCHED_SURROGATE_PIPELINE = 32
SCHED_NO_CLUSTER = 64
SCHED_FOUR_CTAS = 128
SCHED_WARM_STAGED = 256
SCHED_GLOBAL_MEMORY = 512


class ffsrl_info(ctypes.Structure):
    _fields_ = [("n_env", ctypes.c_int32), ("n_meshes", ctypes.c_int32), ("obs_dim", ctypes.c_int32),
                ("max_verts", ctypes.c_int32), ("total_verts", ctypes.c_int64),
                ("block_threads", ctypes.c_int32), ("resident_envs", ctypes.c_int32),
                ("n_groups", ctypes.c_int32), ("ring_envs", ctypes.c_int32),
                ("envs_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libffsrl.so and declares its signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -m paper_2503_18616_gb300.build); "
                           "there is no CPU fallback")
    L = ctypes.CDLL(path)
    P, I32, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
    L.ffsrl_create.restype = ctypes.c_int
    L.ffsrl_create.argtypes = [P, I32, P, P, I32, P, P, ctypes.POINTER(P)]
    L.ffsrl_reset.restype = ctypes.c_int
    L.ffsrl_reset.argtypes = [P, P, U64]
    L.ffsrl_step.restype = ctypes.c_int
    L.ffsrl_step.argtypes = [P, P, P, P, P]
    L.ffsrl_step_host.restype = ctypes.c_int
    L.ffsrl_step_host.argtypes = [P, P, P, P, P]
    L.ffsrl_sync.restype = ctypes.c_int
    L.ffsrl_sync.argtypes = [P]
    L.ffsrl_destroy.restype = ctypes.c_int
    L.ffsrl_destroy.argtypes = [P]
    L.ffsrl_get_info.restype = ctypes.c_int
    L.ffsrl_get_info.argtypes = [P, P]
    L.ffsrl_last_error.restype = ctypes.c_char_p
    L.ffsrl_last_error.argtypes = []
    L.ffsrl_get_state.restype = ctypes.c_int
    L.ffsrl_get_state.argtypes = [P, P, P, P]
    L.ffsrl_set_state.restype = ctypes.c_int
    L.ffsrl_set_state.argtypes = [P, P, P, P]
    L.ffsrl_get_mesh_table.restype = ctypes.c_int
    L.ffsrl_get_mesh_table.argtypes = [P, I32, I32, P, ctypes.POINTER(ctypes.c_int64)]
    L.ffsrl_get_env_ints.restype = ctypes.c_int
    L.ffsrl_get_env_ints.argtypes = [P, I32, P, P, P, P, P]
    L.ffsrl_step_noalloc.restype = ctypes.c_int
    L.ffsrl_step_noalloc.argtypes = [P, P, P, P, P]
    L.ffsrl_set_network.restype = ctypes.c_int
    L.ffsrl_set_network.argtypes = [P, P, P]
    L.ffsrl_network_forward.restype = ctypes.c_int
    L.ffsrl_network_forward.argtypes = [P, P, P, ctypes.c_int64]
    L.ffsrl_step_surrogate.restype = ctypes.c_int
    L.ffsrl_step_surrogate.argtypes = [P, P, P, P, P, ctypes.c_double, I32, P, P]
    L.ffsrl_record_step.restype = ctypes.c_int
    L.ffsrl_record_step.argtypes = [P, P, I32, P, P, P]
    L.ffsrl_get_rows.restype = ctypes.c_int
    L.ffsrl_get_rows.argtypes = [P, ctypes.POINTER(ctypes.c_int64), P]
    L.ffsrl_get_network.restype = ctypes.c_int
    L.ffsrl_get_network.argtypes = [P, P]
    L.ffsrl_network_gradient.restype = ctypes.c_int
    L.ffsrl_network_gradient.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_float, P, P]
    L.ffsrl_train_network.restype = ctypes.c_int
    L.ffsrl_train_network.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, P]
    L.ffsrl_network_adam_step.restype = ctypes.c_int
    L.ffsrl_network_adam_step.argtypes = [P, P, ctypes.c_float]
    L.ffsrl_network_normalisation.restype = ctypes.c_int
    L.ffsrl_network_normalisation.argtypes = [P, P, P, P, ctypes.c_int64, P]
    L.ffsrl_set_env_ids.restype = ctypes.c_int
    L.ffsrl_set_env_ids.argtypes = [P, P]
    L.ffsrl_probe_fp32.restype = ctypes.c_int
    L.ffsrl_probe_fp32.argtypes = [I32, P, P]
    L.ffsrl_probe_smem.restype = ctypes.c_int
    L.ffsrl_probe_smem.argtypes = [I32, P, P]
    L.ffsrl_set_clamp_angles.restype = ctypes.c_int
    L.ffsrl_set_clamp_angles.argtypes = [P, P]
    L.ffsrl_get_grasp.restype = ctypes.c_int
    L.ffsrl_get_grasp.argtypes = [P, P]
    L.ffsrl_set_surrogate_envs.restype = ctypes.c_int
    L.ffsrl_set_surrogate_envs.argtypes = [P, P, ctypes.c_double, I32, P]
    _lib = L
    return L


def _check(rc: int) -> None:
    if rc != FFSRL_OK:
        raise FfsrlError(rc, load_library().ffsrl_last_error().decode())


def _np_ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _dptr(t) -> ctypes.c_void_p | None:
    """Device pointer of a contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def probe_fp32(repeats: int = 5) -> tuple[float, float]:
    """ffsrl_probe_fp32 on the current device: (TFLOP/s, ms of the best launch)."""
    L = load_library()
    r, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(L.ffsrl_probe_fp32(int(repeats), ctypes.byref(r), ctypes.byref(ms)))
    return r.value, ms.value


def probe_smem(repeats: int = 5) -> tuple[float, float]:
    """ffsrl_probe_smem on the current device: (GB/s, ms of the best launch)."""
    L = load_library()
    r, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(L.ffsrl_probe_smem(int(repeats), ctypes.byref(r), ctypes.byref(ms)))
    return r.value, ms.value


def make_params(d: dict, block_threads: int = 0, schedule_flags: int = 0) -> ffsrl_params:
    p = ffsrl_params()
    p.dt = d["dt"]
    p.substeps = d["substeps"]
    p.iterations = d["iterations"]
    p.gravity[:] = [float(g) for g in d["gravity"]]
    p.compliance_dist = d["alpha_d"]
    p.compliance_vol = d["alpha_v"]
    p.tool_radius = d["radius"]
    p.action_scale = d["action_scale"]
    p.tool_margin_xy = d["margin_xy"]
    p.tool_margin_below = d["margin_below"]
    p.tool_margin_above = d["margin_above"]
    p.w_l, p.w_d, p.w_s = d["w_l"], d["w_d"], d["w_s"]
    p.success_dist = d["success_dist"]
    p.n_obs_verts = d["n_obs"]
    p.max_steps = d["max_steps"]
    p.block_threads = block_threads
    p.schedule_flags = schedule_flags
    p.solver = int(d.get("solver", 0))
    p.auto_reset = int(d.get("auto_reset", 0))
    p.tool_model = int(d.get("tool_model", 0))
    for k in ("rcm_height", "shaft_radius", "clamp_length", "clamp_radius", "clamp_angle", "grasp_radius",
              "conn_radius"):
        setattr(p, k, float(d.get(k, 0.0)))
    return p


class Sim:
    """Batched simulator handle (one ffsrl_sim)."""

    def __init__(self, meshes, params: dict, n_env: int, env_mesh=None, env_compliance=None,
                 stream=None, block_threads: int = 0, schedule_flags: int = 0):
        import torch

        self._torch = torch
        L = load_library()
        self._L = L
        self.params = dict(params)
        self._keep = []
        arr = (ffsrl_mesh * len(meshes))()
        for i, (rest, inv_mass, tets) in enumerate(meshes):
            r = np.ascontiguousarray(rest, dtype=np.float64).reshape(-1, 3)
            w = np.ascontiguousarray(inv_mass, dtype=np.float64).reshape(-1)
            t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
            self._keep += [r, w, t]
            arr[i].n_verts, arr[i].n_tets = len(r), len(t)
            arr[i].rest_pos, arr[i].inv_mass, arr[i].tets = r.ctypes.data, w.ctypes.data, t.ctypes.data
        em = None
        if env_mesh is not None:
            em = np.ascontiguousarray(env_mesh, dtype=np.int32)
            self._keep.append(em)
        ec = None
        if env_compliance is not None:
            ec = np.ascontiguousarray(env_compliance, dtype=np.float64)
            self._keep.append(ec)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p = make_params(params, block_threads, schedule_flags)
        h = ctypes.c_void_p()
        _check(L.ffsrl_create(arr, len(meshes), _np_ptr(em) if em is not None else None,
                              _np_ptr(ec) if ec is not None else None, n_env, ctypes.byref(p),
                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h
        info = ffsrl_info()
        _check(L.ffsrl_get_info(self._h, ctypes.byref(info)))
        self.n_env = info.n_env
        self.obs_dim = info.obs_dim
        self.total_verts = info.total_verts
        self.block_threads = info.block_threads
        self.resident_envs = info.resident_envs
        self.n_groups = info.n_groups
        self.ring_envs = info.ring_envs
        self.envs_per_cta = info.envs_per_cta
        self.ctas_per_sm = info.ctas_per_sm
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self) -> None:
        if getattr(self, "_h", None):
            _check(self._L.ffsrl_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- hot path ----------------------------------------------------------
    def reset(self, seed: int = 0, mask=None) -> None:
        _check(self._L.ffsrl_reset(self._h, _dptr(mask), int(seed)))

    def step(self, actions=None, obs=None, reward=None, done=None):
        """One step; allocates missing outputs. Returns (obs, reward, done)."""
        torch = self._torch
        if obs is None:
            obs = torch.empty((self.n_env, self.obs_dim), dtype=torch.float32, device=self.device)
        if reward is None:
            reward = torch.empty(self.n_env, dtype=torch.float32, device=self.device)
        if done is None:
            done = torch.empty(self.n_env, dtype=torch.uint8, device=self.device)
        _check(self._L.ffsrl_step(self._h, _dptr(actions), _dptr(obs), _dptr(reward), _dptr(done)))
        return obs, reward, done

    def step_into(self, actions, obs, reward, done) -> None:
        """ffsrl_step on preallocated tensors (any may be None)."""
        _check(self._L.ffsrl_step(self._h, _dptr(actions), _dptr(obs), _dptr(reward), _dptr(done)))

    def step_host(self, actions=None, obs=None, reward=None, done=None):
        """ffsrl_step_host on numpy buffers (allocated when missing)."""
        if obs is None:
            obs = np.empty((self.n_env, self.obs_dim), dtype=np.float32)
        if reward is None:
            reward = np.empty(self.n_env, dtype=np.float32)
        if done is None:
            done = np.empty(self.n_env, dtype=np.uint8)
        a = None
        if actions is not None:
            a = np.ascontiguousarray(actions, dtype=np.float32).reshape(self.n_env, 3)
        _check(self._L.ffsrl_step_host(self._h, _np_ptr(a) if a is not None else None, _np_ptr(obs),
                                       _np_ptr(reward), _np_ptr(done)))
        return obs, reward, done

    def pinned_host_buffers(self):
        """Page-locked numpy buffers (actions [n_env][3], obs, reward, done)
        for step_host, which then copies to and from them directly."""
        torch = self._torch
        t = (torch.empty((self.n_env, 3), dtype=torch.float32, pin_memory=True),
             torch.empty((self.n_env, self.obs_dim), dtype=torch.float32, pin_memory=True),
             torch.empty(self.n_env, dtype=torch.float32, pin_memory=True),
             torch.empty(self.n_env, dtype=torch.uint8, pin_memory=True))
        self._keep_pinned = getattr(self, "_keep_pinned", []) + [t]
        return tuple(x.numpy() for x in t)

    def step_noalloc(self, actions, x, v, tool) -> None:
        """ffsrl_step_noalloc: one step of the caller's packed state tensors
        (x, v [total_verts][3] float32, tool [n_env][3] float64, updated in
        place) with this sim's meshes; allocates nothing."""
        _check(self._L.ffsrl_step_noalloc(self._h, _dptr(actions), _dptr(x), _dptr(v), _dptr(tool)))

    # -- warm-start network ---------------------------------------------------
    def set_network(self, params: dict, in_mean, in_std, out_mean, out_std) -> None:
        """Installs float32 master weights (dict W1, b1, W2, b2, W3, b3) and the normalisation."""
        flat = np.concatenate([np.asarray(params[k], np.float32).reshape(-1)
                               for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
        norm = np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in (in_mean, in_std, out_mean, out_std)])
        assert flat.size == NET_PARAMS and norm.size == NET_NORM
        _check(self._L.ffsrl_set_network(self._h, _np_ptr(flat), _np_ptr(norm)))

    def get_network(self) -> dict:
        flat = np.zeros(NET_PARAMS, np.float32)
        _check(self._L.ffsrl_get_network(self._h, _np_ptr(flat)))
        out, o = {}, 0
        for k, shape in (("W1", (64, 15)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (3, 64)),
                         ("b3", (3,))):
            n = int(np.prod(shape))
            out[k] = flat[o:o + n].reshape(shape).astype(np.float64)
            o += n
        return out

    def network_gradient(self, features, targets, row_weight, weight_sum: float):
        """(gradient dict, weighted sum of squared errors) of one batch."""
        torch = self._torch
        g = torch.zeros(NET_PARAMS, dtype=torch.float32, device=features.device)
        loss = torch.zeros(1, dtype=torch.float32, device=features.device)
        _check(self._L.ffsrl_network_gradient(self._h, _dptr(features), _dptr(targets), _dptr(row_weight),
                                              int(features.shape[0]), float(weight_sum), _dptr(g), _dptr(loss)))
        flat = g.cpu().numpy().astype(np.float64)
        out, o = {}, 0
        for k, shape in (("W1", (64, 15)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (3, 64)),
                         ("b3", (3,))):
            n = int(np.prod(shape))
            out[k] = flat[o:o + n].reshape(shape)
            o += n
        return out, float(loss.item())

    def train_network(self, features, targets, row_weight, weight_sum: float, lr: float, loss=None):
        _check(self._L.ffsrl_train_network(self._h, _dptr(features), _dptr(targets), _dptr(row_weight),
                                           int(features.shape[0]), float(weight_sum), float(lr), _dptr(loss)))

    def network_adam_step(self, grad, lr: float) -> None:
        """One Adam step of the master parameters on a device gradient
        (float32 tensor [NET_PARAMS] in the parameter layout)."""
        _check(self._L.ffsrl_network_adam_step(self._h, _dptr(grad), float(lr)))

    def network_normalisation(self, features, targets, row_weight):
        """Frozen normalisation of a batch computed on the device:
        (in_mean[15], in_std[15], out_mean[3], out_std[3]) as float64 arrays."""
        out = np.zeros(NET_NORM, np.float32)
        f = features.reshape(-1, 16)
        t = targets.reshape(-1, 4)
        w = row_weight.reshape(-1)
        if not (f.shape[0] == t.shape[0] == w.shape[0]):
            raise ValueError("features, targets and row weights need the same number of rows")
        _check(self._L.ffsrl_network_normalisation(self._h, _dptr(f), _dptr(t), _dptr(w), int(f.shape[0]),
                                                   _np_ptr(out)))
        o = out.astype(np.float64)
        return o[0:15], o[15:30], o[30:33], o[33:36]

    def network_forward(self, features, out=None):
        """features: CUDA tensor [rows][16] float32 -> output [rows][4]."""
        torch = self._torch
        if out is None:
            out = torch.empty((features.shape[0], 4), dtype=torch.float32, device=features.device)
        _check(self._L.ffsrl_network_forward(self._h, _dptr(features), _dptr(out), int(features.shape[0])))
        return out

    def rows(self):
        """(n_rows, row offset of each env) of per-vertex row buffers."""
        n = ctypes.c_int64(0)
        off = np.zeros(self.n_env, np.int32)
        _check(self._L.ffsrl_get_rows(self._h, ctypes.byref(n), _np_ptr(off)))
        return int(n.value), off

    def step_surrogate(self, threshold: float, n_full: int, actions=None, obs=None, reward=None, done=None,
                       fallbacks=None, residual=None):
        torch = self._torch
        if obs is None:
            obs = torch.empty((self.n_env, self.obs_dim), dtype=torch.float32, device=self.device)
        if reward is None:
            reward = torch.empty(self.n_env, dtype=torch.float32, device=self.device)
        if done is None:
            done = torch.empty(self.n_env, dtype=torch.uint8, device=self.device)
        _check(self._L.ffsrl_step_surrogate(self._h, _dptr(actions), _dptr(obs), _dptr(reward), _dptr(done),
                                            float(threshold), int(n_full), _dptr(fallbacks), _dptr(residual)))
        return obs, reward, done

    def set_surrogate_envs(self, mask, threshold: float = float("inf"), n_full: int = 10, fallbacks=None) -> None:
        """Mixed rollout: envs with a non-zero mask byte take the warm-start
        step inside step()/step_host(); mask None switches back to plain."""
        if mask is None:
            _check(self._L.ffsrl_set_surrogate_envs(self._h, None, 0.0, 1, None))
            return
        m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, dtype=np.uint8)
        if m.size != self.n_env:
            raise ValueError("mask needs one byte per env")
        self._mix_keep = fallbacks
        _check(self._L.ffsrl_set_surrogate_envs(self._h, _np_ptr(m), float(threshold), int(n_full),
                                                _dptr(fallbacks)))

    def set_env_ids(self, ids) -> None:
        """Global ids of the envs' counter-based draws (None: 0 .. n_env-1);
        call before reset."""
        if ids is None:
            _check(self._L.ffsrl_set_env_ids(self._h, None))
            return
        a = np.ascontiguousarray(np.asarray(ids).reshape(-1), dtype=np.int64)
        if a.size != self.n_env:
            raise ValueError("need one id per env")
        _check(self._L.ffsrl_set_env_ids(self._h, _np_ptr(a)))

    def set_clamp_angles(self, angles) -> None:
        """Grasper clamp openings (radians, float32 device tensor [n_env])."""
        self._keep_clamp = angles
        _check(self._L.ffsrl_set_clamp_angles(self._h, _dptr(angles)))

    def grasp(self) -> np.ndarray:
        """Grasped vertex of every env (-1: none)."""
        out = np.zeros(self.n_env, np.int32)
        _check(self._L.ffsrl_get_grasp(self._h, _np_ptr(out)))
        return out

    def record_step(self, n_full: int, actions=None, features=None, targets=None, residual=None, want=True):
        """Full-solve step; returns (features [S][rows][16], targets [S][rows][4]) unless want=False."""
        torch = self._torch
        n, _ = self.rows()
        S = self.params["substeps"]
        if want and features is None:
            features = torch.empty((S, n, 16), dtype=torch.float32, device=self.device)
        if want and targets is None:
            targets = torch.empty((S, n, 4), dtype=torch.float32, device=self.device)
        _check(self._L.ffsrl_record_step(self._h, _dptr(actions), int(n_full), _dptr(features), _dptr(targets),
                                         _dptr(residual)))
        return features, targets

    def sync(self) -> None:
        _check(self._L.ffsrl_sync(self._h))

    # -- state access ---------------------------------------------------------
    def get_state(self):
        torch = self._torch
        x = torch.empty((self.total_verts, 3), dtype=torch.float32, device=self.device)
        v = torch.empty_like(x)
        tool = torch.empty((self.n_env, 3), dtype=torch.float64, device=self.device)
        _check(self._L.ffsrl_get_state(self._h, _dptr(x), _dptr(v), _dptr(tool)))
        return x, v, tool

    def set_state(self, x=None, v=None, tool=None) -> None:
        _check(self._L.ffsrl_set_state(self._h, _dptr(x), _dptr(v), _dptr(tool)))

    def mesh_table(self, name: str, mesh: int = 0) -> np.ndarray:
        n = ctypes.c_int64(0)
        _check(self._L.ffsrl_get_mesh_table(self._h, mesh, TABLES[name], None, ctypes.byref(n)))
        out = np.zeros(max(n.value, 1), dtype=np.int32)
        _check(self._L.ffsrl_get_mesh_table(self._h, mesh, TABLES[name], _np_ptr(out), ctypes.byref(n)))
        return out[:n.value].copy()

    def env_ints(self, env: int, max_verts: int | None = None) -> dict:
        t = np.zeros(1, np.int32); tgt = np.zeros(1, np.int32); nc = np.zeros(1, np.int32)
        ids = np.zeros(max(self.params["n_obs"], 1), np.int32)
        cont = np.zeros(max_verts or 65536, np.int32)
        _check(self._L.ffsrl_get_env_ints(self._h, env, _np_ptr(t), _np_ptr(tgt), _np_ptr(ids),
                                          _np_ptr(nc), _np_ptr(cont)))
        return {"t": int(t[0]), "target": int(tgt[0]), "obs_ids": ids[:self.params["n_obs"]].copy(),
                "contacts": cont[:int(nc[0])].copy()}
