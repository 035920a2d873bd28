"""Thin ctypes binding over the C ABI of ``include/vine.h``.

Argument marshalling only: every computation happens in ``libvine.so``.
Importing this module loads the library and raises ImportError when it has
not been built (``python -m paper_2509_15180_gb300.build`` or
``__graft_entry__.build()``); there is no fallback.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
pointers are taken with ``.ctypes.data`` / ``.data_ptr()``.  Streams are
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or None (legacy
default stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvine.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libvine.so is not built (%s); run paper_2509_15180_gb300.build.build()" % LIB_PATH)
_lib = C.CDLL(LIB_PATH)

VINE_OK, VINE_EINVAL, VINE_ENOMEM, VINE_ECUDA, VINE_ETIMEOUT, VINE_EBUSY, VINE_ENOTCONVERGED = range(7)
INST_OK, INST_MAXITER, INST_NONFINITE, INST_BADINPUT = range(4)


class vine_params(C.Structure):
    _fields_ = [("w_a", C.c_double), ("w_b", C.c_double), ("w_c", C.c_double), ("eps_crit", C.c_double),
                ("R_c", C.c_double), ("R_act", C.c_double), ("a_spam", C.c_double), ("m_lo", C.c_double),
                ("pen_frac", C.c_double), ("tol", C.c_double), ("fval_eps", C.c_double),
                ("armijo_c1", C.c_double), ("max_iter", C.c_int32), ("discs_per_link", C.c_int32),
                ("max_halvings", C.c_int32), ("mode", C.c_int32), ("gd_alpha", C.c_double),
                ("gd_steps", C.c_int32), ("exact_hessian", C.c_int32), ("broad_phase", C.c_int32),
                ("threads_per_robot", C.c_int32), ("tol_link", C.c_double)]


class vine_batch_desc(C.Structure):
    _fields_ = [("n_inst", C.c_int32), ("mem_is_device", C.c_int32)] + [
        (k, C.c_void_p) for k in ("n_links", "l_seg", "radius", "pressure", "base", "act_ptr", "act_begin",
                                  "act_end", "act_side", "act_pressure", "act_l0", "obs_ptr", "obs_kind",
                                  "obs_cx", "obs_cy", "obs_a", "obs_b")]


class vine_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("robot_link_steps", "steps_converged", "steps_total", "iterations",
                                         "evaluations", "link_evaluations", "pair_tests", "circle_pair_tests",
                                         "gn_fallbacks")] + [
        (k, C.c_int32) for k in ("n_maxiter", "n_nonfinite", "n_badinput", "reserved")] + [
        ("pair_tests_executed", C.c_int64)]


class vine_server_config(C.Structure):
    _fields_ = [("device_mem_budget", C.c_size_t)] + [
        (k, C.c_int32) for k in ("max_slots", "max_links", "max_obs", "max_act", "max_request", "steps_per_tick",
                                 "max_tables", "lanes", "window")]


class vine_request_info(C.Structure):
    _fields_ = [("n_inst", C.c_int32), ("reserved", C.c_int32), ("total_links", C.c_int64),
                ("robot_link_steps", C.c_int64), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class vine_server_stats(C.Structure):
    _fields_ = [("ticks", C.c_int64), ("requests_done", C.c_int64), ("robot_link_steps", C.c_int64),
                ("active_robots", C.c_int32), ("waiting_requests", C.c_int32), ("free_slots", C.c_int32),
                ("max_slots", C.c_int32), ("busy_s", C.c_double)]


class vine_tune_result(C.Structure):
    _fields_ = [("warps_per_cta", C.c_int32), ("list_margin", C.c_float), ("best_ms", C.c_double),
                ("default_ms", C.c_double), ("candidates", C.c_int32), ("sample", C.c_int32),
                ("n_class", C.c_int32), ("adopted", C.c_int32), ("class_threads", C.c_int32 * 3),
                ("class_robots_per_cta", C.c_int32 * 3), ("class_ms", C.c_double * 3)]


_p, _i32, _i64 = C.c_void_p, C.c_int32, C.c_int64
_SIG = {
    "vine_params_default": [_p],
    "vine_batch_create": [_p, _p, _p, _p],
    "vine_batch_reset": [_p, _p],
    "vine_grow_step": [_p, _i32, _p],
    "vine_simulate": [_p, _p],
    "vine_simulate_plain": [_p, _p],
    "vine_get_state": [_p, _p, _p, _p, _p, _p, _p, _p, _p, _i32, _p],
    "vine_get_contacts": [_p, _p, _p, _i32, _i32, _p],
    "vine_get_stats": [_p, _p, _p],
    "vine_batch_info": [_p, _p, _p],
    "vine_batch_launch": [_p, _p, _p, _p],
    "vine_get_tables": [_p, _p, _p, _p, _p, _p],
    "vine_probe_state": [_p, _i32, _i32, _p, C.c_float, _p, _p, _p, _p, _p],
    "vine_get_robot_counters": [_p, _p, _p, _p, _p],
    "vine_spam_tables_noalloc": [_p, _i32, _p, _p, _p, _p],
    "vine_set_actuators": [_p, _p, _p, _p, _i32, _p],
    "vine_set_state": [_p, _p, _p, _p, _i32, _p],
    "vine_relax": [_p, _i32, _p],
    "vine_synthesize": [_p, _p, _p, _i32, _p, _p, _p, _p, _p],
    "vine_spam_samples": [_p, _p, _i32, _p, _p, _p, _p, _p, _p],
    "vine_surrogate_train": [_p, _p, _p, _i32, _i32, C.c_float, _p, _p],
    "vine_surrogate_eval": [_p, _p, _i32, _p, _i32, _p],
    "vine_sst_prune": [_i32, _p, _p, _p, _i32, _p, _p, C.c_float, C.c_float, _p, _p, _i32, _p],
    "vine_sst_select": [_i32, _p, _p, _p, _i32, _p, C.c_float, C.c_float, _p, _i32, _p],
    "vine_autotune": [_p, _i32, _p, _p],
    "vine_batch_classes": [_p, _p, _p, _p, _p, _p, _p],
    "vine_grad": [_p, _p, _p, _p, _p, _p, _p, _i32, _p],
    "vine_grad_path": [_p, _p, _p, _p, _p, _p, _p, _i32, _p],
    "vine_batch_destroy": [_p],
    "vine_server_config_default": [_p],
    "vine_server_create": [_p, _p, _p],
    "vine_serve_submit": [_p, _p, _p],
    "vine_serve_poll": [_p, C.c_uint64, _i32, _p, _p, _p, _p, _p, _p, _p],
    "vine_server_get_stats": [_p, _p],
    "vine_serve_clock": [_p],
    "vine_server_destroy": [_p],
}
for _name, _args in _SIG.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.vine_last_error.restype = C.c_char_p
_lib.vine_last_error.argtypes = []

EXPORTED = list(_SIG) + ["vine_last_error"]


class VineError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.vine_last_error().decode(errors="replace")
        super().__init__("%s failed with status %d: %s" % (where, status, msg))
        self.status = status


def _check(status: int, where: str):
    if status != VINE_OK:
        raise VineError(status, where)


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _ptr(a) -> int | None:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr()) if a.numel() else None
    a = np.asarray(a)
    return int(a.ctypes.data) if a.size else None


def last_error() -> str:
    return _lib.vine_last_error().decode(errors="replace")


def vine_params_default() -> vine_params:
    p = vine_params()
    _check(_lib.vine_params_default(C.byref(p)), "vine_params_default")
    return p


NOALLOC_MAX_TABLES = 64


def vine_spam_tables_noalloc(l0, hdr, knots, params: vine_params | None = None, stream=None):
    """Allocation-free sPAM table build (vine_spam_tables_noalloc).  l0: CUDA
    float64 tensor [n_tab]; hdr: CUDA float32 [n_tab, 4]; knots: CUDA float32
    [n_tab, 256, 2] -- all allocated by the caller."""
    prm = params if params is not None else vine_params_default()
    _check(_lib.vine_spam_tables_noalloc(_ptr(l0), int(l0.numel()), C.byref(prm), _ptr(hdr), _ptr(knots),
                                         _stream(stream)), "vine_spam_tables_noalloc")


# -------------------------------------------------------------------------
# batch
# -------------------------------------------------------------------------
_HOST_DTYPES = dict(n_links=np.int32, l_seg=np.float32, radius=np.float32, pressure=np.float32,
                    base=np.float32, act_ptr=np.int32, act_begin=np.float32, act_end=np.float32,
                    act_side=np.int8, act_pressure=np.float32, act_l0=np.float32, obs_ptr=np.int32,
                    obs_kind=np.uint8, obs_cx=np.float32, obs_cy=np.float32, obs_a=np.float32,
                    obs_b=np.float32)


class Batch:
    """A batch handle: ``vine_batch_create`` on construction,
    ``vine_batch_destroy`` on close()."""

    def __init__(self, scene: dict, params: vine_params | None = None, stream=None):
        keep = {}
        dev = 0
        for k, dt in _HOST_DTYPES.items():
            v = scene[k]
            if hasattr(v, "data_ptr"):  # torch tensor
                dev = 1 if v.is_cuda else dev
                keep[k] = v.contiguous()
            else:
                keep[k] = np.ascontiguousarray(np.asarray(v).reshape(-1), dtype=dt)
        self._keep = keep
        D = vine_batch_desc()
        D.n_inst = int(len(scene["n_links"]))
        D.mem_is_device = dev
        for k in _HOST_DTYPES:
            setattr(D, k, _ptr(keep[k]))
        self.n_inst = D.n_inst
        self.params = params if params is not None else vine_params_default()
        h = C.c_void_p()
        _check(_lib.vine_batch_create(C.byref(D), C.byref(self.params), _stream(stream), C.byref(h)),
               "vine_batch_create")
        self.h = h
        n, tl = C.c_int32(), C.c_int64()
        _check(_lib.vine_batch_info(h, C.byref(n), C.byref(tl)), "vine_batch_info")
        self.total_links = tl.value
        nl = scene["n_links"]
        self.n_links = nl.cpu().numpy() if hasattr(nl, "cpu") else np.asarray(nl)
        ap = scene["act_ptr"]
        self.act_ptr = (ap.cpu().numpy() if hasattr(ap, "cpu") else np.asarray(ap)).astype(np.int64)
        self.n_act = int(self.act_ptr[-1])
        self.offsets = np.concatenate([[0], np.cumsum(self.n_links)]).astype(np.int64)
        self._keep = None  # inputs were copied during create

    def close(self):
        if getattr(self, "h", None):
            _lib.vine_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        _check(_lib.vine_batch_reset(self.h, _stream(stream)), "vine_batch_reset")

    def grow_step(self, n_steps: int = 1, stream=None):
        _check(_lib.vine_grow_step(self.h, int(n_steps), _stream(stream)), "vine_grow_step")

    def launch(self) -> dict:
        """vine_batch_launch: threads per robot, robots per CTA, CTAs."""
        t, w, g = C.c_int32(), C.c_int32(), C.c_int32()
        _check(_lib.vine_batch_launch(self.h, C.byref(t), C.byref(w), C.byref(g)), "vine_batch_launch")
        return dict(threads_per_robot=t.value, robots_per_cta=w.value, grid=g.value)

    def relax(self, fix_length: bool = True, stream=None):
        """vine_relax: re-solve at the present links, no link added."""
        _check(_lib.vine_relax(self.h, int(bool(fix_length)), _stream(stream)), "vine_relax")

    def simulate(self, stream=None):
        _check(_lib.vine_simulate(self.h, _stream(stream)), "vine_simulate")

    def autotune(self, sample: int = 4096, stream=None) -> dict:
        """Time launch configurations on a sample and adopt the fastest
        (vine_autotune); leaves the batch reset."""
        r = vine_tune_result()
        _check(_lib.vine_autotune(self.h, int(sample), _stream(stream), C.byref(r)), "vine_autotune")
        out = {k: getattr(r, k) for k, _ in vine_tune_result._fields_}
        for k in ("class_threads", "class_robots_per_cta", "class_ms"):
            out[k] = list(out[k])[: r.n_class]
        return out

    def classes(self) -> list:
        """vine_batch_classes: per length class (longest robots first) threads
        per robot, robots, robots per CTA, CTAs and the longest robot's links."""
        n = C.c_int32()
        a = [np.zeros(3, np.int32) for _ in range(5)]
        _check(_lib.vine_batch_classes(self.h, C.byref(n), *[_ptr(x) for x in a]), "vine_batch_classes")
        keys = ("threads_per_robot", "robots", "robots_per_cta", "grid", "max_links")
        return [{k: int(x[c]) for k, x in zip(keys, a)} for c in range(n.value)]

    def simulate_plain(self, stream=None):
        _check(_lib.vine_simulate_plain(self.h, _stream(stream)), "vine_simulate_plain")

    def set_actuators(self, pressure, begin, end, stream=None):
        """New actuator pressures (Pa) and spans (link units), [n_act] each:
        numpy arrays (synchronous) or CUDA float32 tensors (async)."""
        dev = int(hasattr(pressure, "is_cuda") and pressure.is_cuda)
        if dev:
            args = [x.contiguous() for x in (pressure, begin, end)]
        else:
            args = [np.ascontiguousarray(np.asarray(x).reshape(-1), np.float32) for x in (pressure, begin, end)]
        for x in args:
            if (x.numel() if dev else x.size) != self.n_act:
                raise ValueError("set_actuators: expected %d values per array" % self.n_act)
        _check(_lib.vine_set_actuators(self.h, _ptr(args[0]), _ptr(args[1]), _ptr(args[2]), dev, _stream(stream)),
               "vine_set_actuators")
        self._act_keep = args  # alive until the async copy has run

    def set_state(self, n_present, theta, l_last, stream=None):
        """Present state to continue growth from (vine_set_state): links
        present [n], joint angles [sum n_links] in the CSR layout of state(),
        distal lengths [n].  numpy arrays (synchronous) or CUDA tensors
        (int32 / float32, async).  Counters are cleared."""
        n, T = self.n_inst, self.total_links
        dev = int(hasattr(theta, "is_cuda") and theta.is_cuda)
        if dev:
            args = [n_present.contiguous(), theta.contiguous(), l_last.contiguous()]
            sizes = [x.numel() for x in args]
        else:
            args = [np.ascontiguousarray(np.asarray(n_present).reshape(-1), np.int32),
                    np.ascontiguousarray(np.asarray(theta).reshape(-1), np.float32),
                    np.ascontiguousarray(np.asarray(l_last).reshape(-1), np.float32)]
            sizes = [x.size for x in args]
        if sizes[0] != n or sizes[2] != n or sizes[1] < T:
            raise ValueError("set_state: expected [%d], [%d] and [%d] values" % (n, T, n))
        _check(_lib.vine_set_state(self.h, _ptr(args[0]), _ptr(args[1]), _ptr(args[2]), dev, _stream(stream)),
               "vine_set_state")
        self._state_keep = args  # alive until the async copy has run

    def grad(self, goal, stream=None) -> dict:
        """Tip-distance cost |p_tip - goal| and its adjoint derivatives at the
        current state (vine_grad).  goal: [n, 2] numpy (host path, returns
        numpy) or CUDA float32 tensor (device path, returns CUDA tensors,
        async)."""
        return self._grad(_lib.vine_grad, "vine_grad", goal, self.n_inst, stream)

    def grad_path(self, path, stream=None) -> dict:
        """Path cost (1/N) sum_k |p_k - q_k|^2 of the link end points against
        targets path [total_links, 2] (robot i's rows at its joint-angle
        offset) and its adjoint derivatives (vine_grad_path); numpy or CUDA
        float32 as grad()."""
        return self._grad(_lib.vine_grad_path, "vine_grad_path", path, max(self.total_links, 1), stream)

    def _grad(self, fn, name, goal, rows, stream):
        n, na = self.n_inst, self.n_act
        if hasattr(goal, "is_cuda") and goal.is_cuda:
            import torch
            g = goal.contiguous()
            out = dict(cost=torch.empty(n, dtype=torch.float64, device=g.device),
                       dP=torch.empty(max(na, 1), dtype=torch.float64, device=g.device),
                       dB=torch.empty(max(na, 1), dtype=torch.float64, device=g.device),
                       dE=torch.empty(max(na, 1), dtype=torch.float64, device=g.device),
                       status=torch.empty(n, dtype=torch.int32, device=g.device))
            dev = 1
        else:
            g = np.ascontiguousarray(np.asarray(goal, np.float32).reshape(-1, 2))
            out = dict(cost=np.zeros(n), dP=np.zeros(max(na, 1)), dB=np.zeros(max(na, 1)), dE=np.zeros(max(na, 1)),
                       status=np.zeros(n, np.int32))
            dev = 0
        if int(np.prod(tuple(g.shape))) < 2 * rows:
            raise ValueError("%s: expected [%d, 2] target points" % (name, rows))
        _check(fn(self.h, _ptr(g), _ptr(out["cost"]), _ptr(out["dP"]), _ptr(out["dB"]), _ptr(out["dE"]),
                  _ptr(out["status"]), dev, _stream(stream)), name)
        for k in ("dP", "dB", "dE"):
            out[k] = out[k][:na]
        return out

    def state(self, stream=None) -> dict:
        """Host copy of the state (synchronises the stream)."""
        n, T = self.n_inst, max(self.total_links, 1)
        out = dict(theta=np.zeros(T, np.float32), l=np.zeros(n, np.float32), pose=np.zeros((T, 3), np.float32),
                   tip=np.zeros((n, 2), np.float32), N=np.zeros(n, np.int32), iters=np.zeros(n, np.int32),
                   resid=np.zeros(n, np.float64), status=np.zeros(n, np.int32))
        _check(_lib.vine_get_state(self.h, _ptr(out["theta"]), _ptr(out["l"]), _ptr(out["pose"]), _ptr(out["tip"]),
                                   _ptr(out["N"]), _ptr(out["iters"]), _ptr(out["resid"]), _ptr(out["status"]), 0,
                                   _stream(stream)), "vine_get_state")
        return out

    def state_device(self, out: dict, stream=None):
        """Writes the state into torch CUDA tensors (async on the stream)."""
        g = lambda k: _ptr(out.get(k))
        _check(_lib.vine_get_state(self.h, g("theta"), g("l"), g("pose"), g("tip"), g("N"), g("iters"),
                                   g("resid"), g("status"), 1, _stream(stream)), "vine_get_state")

    def contacts(self, max_pairs: int = 256, stream=None):
        """(counts[n], pairs[n, max_pairs, 2]) at the current state."""
        counts = np.zeros(self.n_inst, np.int32)
        pairs = np.zeros((self.n_inst, max_pairs, 2), np.int32)
        _check(_lib.vine_get_contacts(self.h, _ptr(counts), _ptr(pairs), int(max_pairs), 0, _stream(stream)),
               "vine_get_contacts")
        return counts, pairs

    def stats(self, stream=None) -> dict:
        s = vine_stats()
        _check(_lib.vine_get_stats(self.h, C.byref(s), _stream(stream)), "vine_get_stats")
        return {k: getattr(s, k) for k, _ in vine_stats._fields_}

    def tables(self) -> dict:
        """Prologue tables as the kernels use them (see vine_get_tables)."""
        nt = C.c_int32()
        _check(_lib.vine_get_tables(self.h, C.byref(nt), None, None, None, None), "vine_get_tables")
        n = nt.value
        hdr = np.zeros((max(n, 1), 4), np.float32)
        kn = np.zeros((max(n, 1), 256, 2), np.float32)
        ut = np.zeros((1025, 2), np.float32)
        cs = np.zeros(4, np.float64)
        _check(_lib.vine_get_tables(self.h, C.byref(nt), _ptr(hdr), _ptr(kn), _ptr(ut), _ptr(cs)),
               "vine_get_tables")
        return dict(n_tab=n, hdr=hdr[:n], knots=kn[:n], utab=ut, consts=cs)

    def probe(self, i: int, theta, l: float):
        """(cost, grad[N+1], step[N+1], residual, l_fixed) at a given state (vine_probe_state)."""
        th = np.ascontiguousarray(theta, dtype=np.float32)
        N = th.size
        J, r, lf = C.c_double(), C.c_double(), C.c_int32()
        g = np.zeros(N + 1, np.float32)
        dx = np.zeros(N + 1, np.float32)
        _check(_lib.vine_probe_state(self.h, int(i), N, _ptr(th), float(l), C.byref(J), _ptr(g), _ptr(dx),
                                     C.byref(r), C.byref(lf)), "vine_probe_state")
        return J.value, g, dx, r.value, bool(lf.value)

    def robot_counters(self, stream=None) -> dict:
        """Per-robot converged steps, evaluations and SM cycles (vine_get_robot_counters)."""
        n = self.n_inst
        out = dict(conv=np.zeros(n, np.int32), evals=np.zeros(n, np.int64), cycles=np.zeros(n, np.int64))
        _check(_lib.vine_get_robot_counters(self.h, _ptr(out["conv"]), _ptr(out["evals"]), _ptr(out["cycles"]),
                                            _stream(stream)), "vine_get_robot_counters")
        return out

    def theta_of(self, st: dict, i: int):
        return st["theta"][self.offsets[i]: self.offsets[i] + st["N"][i]]

    def pose_of(self, st: dict, i: int):
        return st["pose"][self.offsets[i]: self.offsets[i] + st["N"][i]]


# -------------------------------------------------------------------------
# actuator design synthesis (Sec. 4.2)
# -------------------------------------------------------------------------
class vine_synth_spec(C.Structure):
    _fields_ = [("R", C.c_double), ("P_vine", C.c_double), ("l_seg", C.c_double), ("pressures", C.c_void_p),
                ("n_p", C.c_int32), ("l0_min", C.c_double), ("l0_step", C.c_double), ("n_l0", C.c_int32),
                ("tol", C.c_double)]


def synthesize(theta_targets, R: float, P_vine: float, l_seg: float, pressures, l0_min: float, l0_step: float,
               n_l0: int, tol: float, params: vine_params | None = None, stream=None) -> dict:
    """vine_synthesize: per target angle per joint, the chosen pressure index,
    cell-length index (-1: none feasible) and the angle the design holds;
    and the angle of every (pressure, cell length) pair."""
    tg = np.ascontiguousarray(np.asarray(theta_targets, np.float64).reshape(-1))
    pr = np.ascontiguousarray(np.asarray(pressures, np.float64).reshape(-1))
    spec = vine_synth_spec(float(R), float(P_vine), float(l_seg), pr.ctypes.data, pr.size, float(l0_min),
                           float(l0_step), int(n_l0), float(tol))
    n = tg.size
    out = dict(p_index=np.zeros(n, np.int32), l0_index=np.zeros(n, np.int32), theta_eq=np.zeros(n),
               pairs=np.zeros((pr.size, int(n_l0))))
    _check(_lib.vine_synthesize(C.byref(spec), C.byref(params) if params is not None else None, _ptr(tg), n,
                                _ptr(out["p_index"]), _ptr(out["l0_index"]), _ptr(out["theta_eq"]),
                                _ptr(out["pairs"]), _stream(stream)), "vine_synthesize")
    return out


# -------------------------------------------------------------------------
# sPAM surrogate (Sec. 4.3)
# -------------------------------------------------------------------------
class vine_surrogate(C.Structure):
    _fields_ = [("theta", C.c_float * 162), ("in_lo", C.c_float * 2), ("in_scale", C.c_float * 2),
                ("out_scale", C.c_float * 2)]


def _net_struct(net: dict) -> vine_surrogate:
    s = vine_surrogate()
    s.theta[:] = [float(v) for v in np.asarray(net["theta"], np.float32)]
    for k in ("in_lo", "in_scale", "out_scale"):
        getattr(s, k)[:] = [float(v) for v in np.asarray(net[k], np.float32)]
    return s


def spam_samples(m, l0, params: vine_params | None = None, stream=None) -> dict:
    """vine_spam_samples: the exact sPAM model at (m, l0) pairs."""
    m = np.ascontiguousarray(np.asarray(m, np.float64).reshape(-1))
    l0 = np.ascontiguousarray(np.asarray(l0, np.float64).reshape(-1))
    n = m.size
    out = dict(eps=np.zeros(n), phi=np.zeros(n), f=np.zeros(n), saturated=np.zeros(n, np.int32))
    _check(_lib.vine_spam_samples(_ptr(m), _ptr(l0), n, C.byref(params) if params is not None else None,
                                  _ptr(out["eps"]), _ptr(out["phi"]), _ptr(out["f"]), _ptr(out["saturated"]),
                                  _stream(stream)), "vine_spam_samples")
    return out


def surrogate_train(net: dict, inputs, targets, steps: int, lr: float, history: bool = True, stream=None):
    """vine_surrogate_train: returns (trained net dict, loss history or None)."""
    s = _net_struct(net)
    x = np.ascontiguousarray(np.asarray(inputs, np.float64).reshape(-1, 2))
    t = np.ascontiguousarray(np.asarray(targets, np.float64).reshape(-1, 2))
    hist = np.zeros(max(int(steps), 1), np.float32) if history else None
    _check(_lib.vine_surrogate_train(C.byref(s), _ptr(x), _ptr(t), x.shape[0], int(steps), float(lr),
                                     _ptr(hist) if history else None, _stream(stream)), "vine_surrogate_train")
    out = dict(net, theta=np.array(s.theta[:], np.float32))
    return out, (hist[: int(steps)] if history else None)


def surrogate_eval(net: dict, inputs, stream=None):
    """vine_surrogate_eval: (m, phi) per input row; numpy in/out, or CUDA
    float64 tensors [n, 2] (async)."""
    s = _net_struct(net)
    if hasattr(inputs, "is_cuda") and inputs.is_cuda:
        import torch
        x = inputs.contiguous()
        out = torch.empty_like(x)
        _check(_lib.vine_surrogate_eval(C.byref(s), _ptr(x), x.shape[0], _ptr(out), 1, _stream(stream)),
               "vine_surrogate_eval")
        return out
    x = np.ascontiguousarray(np.asarray(inputs, np.float64).reshape(-1, 2))
    out = np.zeros_like(x)
    _check(_lib.vine_surrogate_eval(C.byref(s), _ptr(x), x.shape[0], _ptr(out), 0, _stream(stream)),
           "vine_surrogate_eval")
    return out


# -------------------------------------------------------------------------
# planner tree operations (Sec. 5.2, Algorithm 2)
# -------------------------------------------------------------------------
def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def sst_prune(old_pose, old_cost, old_active, new_pose, new_cost, radius: float, rho: float, stream=None):
    """vine_sst_prune.  Poses [n, 3] float32, costs [n] float64, active [n]
    uint8: numpy arrays (returns numpy, synchronous) or CUDA tensors
    (returns CUDA uint8 tensors, async).  Returns (keep[n_new],
    deactivate[n_old])."""
    if _is_cuda(new_pose) or _is_cuda(old_pose):
        import torch
        dev = new_pose.device if _is_cuda(new_pose) else old_pose.device
        a = [old_pose.contiguous(), old_cost.contiguous(), old_active.contiguous(), new_pose.contiguous(),
             new_cost.contiguous()]
        n_old, n_new = a[1].numel(), a[4].numel()
        keep = torch.empty(n_new, dtype=torch.uint8, device=dev)
        deact = torch.empty(n_old, dtype=torch.uint8, device=dev)
        flag = 1
    else:
        a = [np.ascontiguousarray(np.asarray(old_pose, np.float32).reshape(-1, 3)),
             np.ascontiguousarray(np.asarray(old_cost, np.float64).reshape(-1)),
             np.ascontiguousarray(np.asarray(old_active, np.uint8).reshape(-1)),
             np.ascontiguousarray(np.asarray(new_pose, np.float32).reshape(-1, 3)),
             np.ascontiguousarray(np.asarray(new_cost, np.float64).reshape(-1))]
        n_old, n_new = a[1].size, a[4].size
        keep = np.zeros(n_new, np.uint8)
        deact = np.zeros(n_old, np.uint8)
        flag = 0
    _check(_lib.vine_sst_prune(n_old, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), n_new, _ptr(a[3]), _ptr(a[4]),
                               float(radius), float(rho), _ptr(keep), _ptr(deact), flag, _stream(stream)),
           "vine_sst_prune")
    return keep, deact


def sst_select(pose, cost, active, samples, delta: float, rho: float, stream=None):
    """vine_sst_select.  Returns the chosen node per sample (int32; -1 when no
    node is active): numpy for numpy inputs, a CUDA tensor for CUDA inputs."""
    if _is_cuda(samples):
        import torch
        a = [pose.contiguous(), cost.contiguous(), active.contiguous(), samples.contiguous()]
        n_nodes, n_s = a[1].numel(), a[3].numel() // 3
        out = torch.empty(n_s, dtype=torch.int32, device=samples.device)
        flag = 1
    else:
        a = [np.ascontiguousarray(np.asarray(pose, np.float32).reshape(-1, 3)),
             np.ascontiguousarray(np.asarray(cost, np.float64).reshape(-1)),
             np.ascontiguousarray(np.asarray(active, np.uint8).reshape(-1)),
             np.ascontiguousarray(np.asarray(samples, np.float32).reshape(-1, 3))]
        n_nodes, n_s = a[1].size, a[3].shape[0]
        out = np.zeros(n_s, np.int32)
        flag = 0
    _check(_lib.vine_sst_select(n_nodes, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), n_s, _ptr(a[3]), float(delta),
                                float(rho), _ptr(out), flag, _stream(stream)), "vine_sst_select")
    return out


# -------------------------------------------------------------------------
# serving loop
# -------------------------------------------------------------------------
def serve_clock() -> float:
    """The server clock (seconds, monotonic) of t_submit / t_admit / t_done."""
    t = C.c_double()
    _check(_lib.vine_serve_clock(C.byref(t)), "vine_serve_clock")
    return t.value


def _host_desc(scene: dict):
    keep = {k: np.ascontiguousarray(np.asarray(scene[k]).reshape(-1), dtype=dt) for k, dt in _HOST_DTYPES.items()}
    D = vine_batch_desc()
    D.n_inst = int(len(keep["n_links"]))
    D.mem_is_device = 0
    for k in _HOST_DTYPES:
        setattr(D, k, _ptr(keep[k]))
    return D, keep


class Server:
    """A serving loop (vine_server_create); config keys as vine_server_config."""

    def __init__(self, params: vine_params | None = None, **config):
        cfg = vine_server_config()
        _check(_lib.vine_server_config_default(C.byref(cfg)), "vine_server_config_default")
        for k, v in config.items():
            setattr(cfg, k, v)
        self.params = params if params is not None else vine_params_default()
        h = C.c_void_p()
        _check(_lib.vine_server_create(C.byref(self.params), C.byref(cfg), C.byref(h)), "vine_server_create")
        self.h = h
        self._sizes = {}

    def submit(self, scene: dict):
        """Request id, or None when the server is full (VINE_EBUSY: retry later)."""
        D, keep = _host_desc(scene)
        rid = C.c_uint64()
        st = _lib.vine_serve_submit(self.h, C.byref(D), C.byref(rid))
        if st == VINE_EBUSY:
            return None
        _check(st, "vine_serve_submit")
        self._sizes[rid.value] = (D.n_inst, int(keep["n_links"].sum()))
        return rid.value

    def poll(self, rid: int, timeout_us: int = 0):
        """Result dict of a finished request (then released), or None if it is
        not finished within timeout_us."""
        n, T = self._sizes.get(rid, (1, 1))  # unknown ids are reported by the library
        out = dict(theta=np.zeros(max(T, 1), np.float32), l=np.zeros(n, np.float32), tip=np.zeros((n, 2), np.float32),
                   N=np.zeros(n, np.int32), status=np.zeros(n, np.int32), iters=np.zeros(n, np.int32))
        info = vine_request_info()
        st = _lib.vine_serve_poll(self.h, C.c_uint64(rid), int(timeout_us), C.byref(info), _ptr(out["theta"]),
                                  _ptr(out["l"]), _ptr(out["tip"]), _ptr(out["N"]), _ptr(out["status"]),
                                  _ptr(out["iters"]))
        if st == VINE_ETIMEOUT:
            return None
        self._sizes.pop(rid, None)
        _check(st, "vine_serve_poll")
        out["theta"] = out["theta"][:T]
        out.update(rls=info.robot_link_steps, t_submit=info.t_submit, t_admit=info.t_admit, t_done=info.t_done)
        return out

    def stats(self) -> dict:
        s = vine_server_stats()
        _check(_lib.vine_server_get_stats(self.h, C.byref(s)), "vine_server_get_stats")
        return {k: getattr(s, k) for k, _ in vine_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib.vine_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
