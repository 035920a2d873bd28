"""FP64 CPU oracle for the vine-robot growth step (arXiv 2509.15180).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product package never
imports this module, and this module imports nothing from the product
package.  The arithmetic lives in ``vine_oracle.c`` (plain C, double
precision); this file only marshals numpy arrays through ctypes.

Scene dictionaries come from the seeded generator (``paper_2509_15180_gb300.scenes``),
which holds no model arithmetic.  Their float32 values are widened to
float64 here, so that both sides start from bit-identical inputs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vine_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libvine_oracle.so")
NKNOT = 256

STATUS_OK, STATUS_MAXITER, STATUS_NONFINITE, STATUS_BADINPUT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               _SRC, "-o", _LIB, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class Params(C.Structure):
    _fields_ = [("w_a", C.c_double), ("w_b", C.c_double), ("w_c", C.c_double),
                ("eps_crit", C.c_double), ("R_c", C.c_double), ("R_act", C.c_double),
                ("a_spam", C.c_double), ("m_lo", C.c_double), ("pen_frac", C.c_double),
                ("tol", C.c_double), ("fval_eps", C.c_double), ("armijo_c1", C.c_double),
                ("max_iter", C.c_int32), ("discs_per_link", C.c_int32),
                ("max_halvings", C.c_int32), ("exact_hessian", C.c_int32), ("mode", C.c_int32),
                ("gd_steps", C.c_int32), ("gd_alpha", C.c_double), ("tol_link", C.c_double)]


class _Batch(C.Structure):
    _fields_ = [("n_inst", C.c_int32),
                ("n_links", C.c_void_p), ("l_seg", C.c_void_p), ("radius", C.c_void_p),
                ("pressure", C.c_void_p), ("base", C.c_void_p),
                ("act_ptr", C.c_void_p), ("act_begin", C.c_void_p), ("act_end", C.c_void_p),
                ("act_side", C.c_void_p), ("act_pressure", C.c_void_p), ("act_l0", C.c_void_p),
                ("obs_ptr", C.c_void_p), ("obs_kind", C.c_void_p), ("obs_cx", C.c_void_p),
                ("obs_cy", C.c_void_p), ("obs_a", C.c_void_p), ("obs_b", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        d, p, i = C.c_double, C.c_void_p, C.c_int
        L.orc_params_default.argtypes = [p]
        L.orc_ellip_F.restype = d
        L.orc_ellip_F.argtypes = [d, d]
        L.orc_ellip_E.restype = d
        L.orc_ellip_E.argtypes = [d, d]
        L.orc_spam_eval.argtypes = [p, d, d, p, p, p, p]
        L.orc_spam_table.argtypes = [p, d, p, p, p]
        L.orc_table_eval.argtypes = [d, d, p, d, p, p, p]
        L.orc_wrinkle.argtypes = [d, d, p, p, p]
        L.orc_tables_create.restype = p
        L.orc_tables_create.argtypes = [p, p]
        L.orc_tables_free.argtypes = [p]
        L.orc_tables_count.restype = i
        L.orc_tables_count.argtypes = [p]
        L.orc_tables_get.argtypes = [p, i, p, p, p, p]
        L.orc_energy.restype = d
        L.orc_energy.argtypes = [p, p, p, i, i, p, d, p, p]
        L.orc_energy_exact.restype = d
        L.orc_energy_exact.argtypes = [p, p, p, i, i, p, d, p, p]
        L.orc_solve.restype = i
        L.orc_solve.argtypes = [p, p, p, i, i, p, p, p, p, i]
        L.orc_poses.argtypes = [p, p, p, i, i, p, d, p, p, p]
        L.orc_gaps.argtypes = [p, p, p, i, i, p, d, p]
        L.orc_sdf.restype = d
        L.orc_sdf.argtypes = [p, i, d, d, p, p]
        L.orc_gn_step.restype = i
        L.orc_gn_step.argtypes = [p, p, p, i, i, p, d, p, p, p, p, i]
        L.orc_grad.restype = i
        L.orc_grad.argtypes = [p, p, p, i, i, p, d, d, d, p, p, p, p]
        L.orc_grad_path.restype = i
        L.orc_grad_path.argtypes = [p, p, p, i, i, p, d, p, p, p, p, p, p]
        L.orc_set_trace.argtypes = [i]
        L.orc_run.restype = i
        L.orc_run.argtypes = [p, p, p, i, p, p, p, p, p, p, p, p, p, i]
        L.orc_relax.restype = i
        L.orc_relax.argtypes = [p, p, p, i, p, p, p, p, p, p, p, p, p, i]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_params(**over) -> Params:
    P = Params()
    lib().orc_params_default(C.byref(P))
    for k, v in over.items():
        setattr(P, k, v)
    return P


# --------------------------------------------------------------------------
# model components (for the pins)
# --------------------------------------------------------------------------
def ellip_F(phi: float, m: float) -> float:
    return lib().orc_ellip_F(float(phi), float(m))


def ellip_E(phi: float, m: float) -> float:
    return lib().orc_ellip_E(float(phi), float(m))


def spam_eval(m: float, l0: float, params: Params | None = None):
    """(eps, f = F_t / P_act, phi_Rc, saturated) at contraction parameter m."""
    P = params or default_params()
    e, f, ph, s = C.c_double(), C.c_double(), C.c_double(), C.c_int()
    rc = lib().orc_spam_eval(C.byref(P), float(m), float(l0), C.byref(e), C.byref(f), C.byref(ph), C.byref(s))
    if rc != 0:
        raise ValueError("sPAM model has no finite solution at m=%g" % m)
    return e.value, f.value, ph.value, bool(s.value)


def spam_table(l0: float, params: Params | None = None):
    """(eps_lo, eps_hi, f[NKNOT]) for cell length l0."""
    P = params or default_params()
    f = np.zeros(NKNOT)
    lo, hi = C.c_double(), C.c_double()
    rc = lib().orc_spam_table(C.byref(P), float(l0), C.byref(lo), C.byref(hi), _ptr(f))
    if rc != 0:
        raise ValueError("table build failed")
    return lo.value, hi.value, f


def table_eval(eps_lo: float, eps_hi: float, f: np.ndarray, eps: float):
    """(f, df/deps, integral_0^eps f) of the piecewise-linear interpolant."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().orc_table_eval(float(eps_lo), float(eps_hi), _ptr(f), float(eps), C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def wrinkle(theta: float, eps_c: float = 0.01, energy: bool = True):
    """(M, dM/dtheta, integral_0^theta M), all divided by pi P R^3 (the
    integral is None unless energy=True)."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().orc_wrinkle(float(theta), float(eps_c), C.byref(a), C.byref(b), C.byref(c) if energy else None)
    return a.value, b.value, (c.value if energy else None)


# --------------------------------------------------------------------------
# batch-level access
# --------------------------------------------------------------------------
class Oracle:
    """FP64 oracle over a scene dictionary (CSR layout, see scenes.py)."""

    def __init__(self, scene: dict, params: Params | None = None):
        self.P = params or default_params()
        self.fix_length = False  # solve / gn_step: hold the distal length fixed (relaxation)
        self.n = int(len(scene["n_links"]))
        f64 = lambda k: np.ascontiguousarray(scene[k], dtype=np.float64)
        i32 = lambda k: np.ascontiguousarray(scene[k], dtype=np.int32)
        self._keep = dict(
            n_links=i32("n_links"), l_seg=f64("l_seg"), radius=f64("radius"), pressure=f64("pressure"),
            base=np.ascontiguousarray(np.asarray(scene["base"], dtype=np.float64).reshape(-1)),
            act_ptr=i32("act_ptr"), act_begin=f64("act_begin"), act_end=f64("act_end"),
            act_side=i32("act_side"), act_pressure=f64("act_pressure"), act_l0=f64("act_l0"),
            obs_ptr=i32("obs_ptr"), obs_kind=i32("obs_kind"), obs_cx=f64("obs_cx"), obs_cy=f64("obs_cy"),
            obs_a=f64("obs_a"), obs_b=f64("obs_b"))
        # empty arrays still need a valid pointer
        for k, v in self._keep.items():
            if v.size == 0:
                self._keep[k] = np.zeros(1, dtype=v.dtype)
        B = _Batch()
        B.n_inst = self.n
        for k, v in self._keep.items():
            setattr(B, k, v.ctypes.data)
        self.B = B
        self.T = lib().orc_tables_create(C.byref(self.P), C.byref(self.B))
        if not self.T:
            raise ValueError("sPAM table build failed")
        self.n_links = self._keep["n_links"]
        self.off = np.concatenate([[0], np.cumsum(self.n_links)]).astype(np.int64)

    def __del__(self):
        try:
            if getattr(self, "T", None):
                lib().orc_tables_free(self.T)
        except Exception:
            pass

    def tables(self):
        out = []
        for t in range(lib().orc_tables_count(self.T)):
            l0, lo, hi = C.c_double(), C.c_double(), C.c_double()
            f = np.zeros(NKNOT)
            lib().orc_tables_get(self.T, t, C.byref(l0), C.byref(lo), C.byref(hi), _ptr(f))
            out.append((l0.value, lo.value, hi.value, f))
        return out

    def energy(self, i: int, theta, l: float, hessian: bool = True):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        N = th.size
        g = np.zeros(N + 1)
        H = np.zeros((N + 1) * (N + 1)) if hessian else None
        J = lib().orc_energy(C.byref(self.P), C.byref(self.B), self.T, int(i), N, _ptr(th), float(l), _ptr(g),
                             _ptr(H) if hessian else None)
        return J, g, (H.reshape(N + 1, N + 1) if hessian else None)

    def hessian_exact(self, i: int, theta, l: float):
        """Exact Hessian of J (contact curvature and load terms included)."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        N = th.size
        g = np.zeros(N + 1)
        H = np.zeros((N + 1) * (N + 1))
        lib().orc_energy_exact(C.byref(self.P), C.byref(self.B), self.T, int(i), N, _ptr(th), float(l), _ptr(g),
                               _ptr(H))
        return H.reshape(N + 1, N + 1)

    def solve(self, i: int, theta, l: float):
        th = np.array(theta, dtype=np.float64)
        lv = C.c_double(float(l))
        it, r = C.c_int(), C.c_double()
        st = lib().orc_solve(C.byref(self.P), C.byref(self.B), self.T, int(i), th.size, _ptr(th), C.byref(lv),
                             C.byref(it), C.byref(r), int(self.fix_length))
        return th, lv.value, it.value, r.value, st

    def gn_step(self, i: int, theta, l: float):
        """(dx[N+1], residual, J, lfix): the solver's Newton step at a fixed state
        (exact Hessian when positive definite, else Gauss-Newton)."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        N = th.size
        dx = np.zeros(N + 1)
        r, J, lf = C.c_double(), C.c_double(), C.c_int()
        rc = lib().orc_gn_step(C.byref(self.P), C.byref(self.B), self.T, int(i), N, _ptr(th), float(l), _ptr(dx),
                               C.byref(r), C.byref(J), C.byref(lf), int(self.fix_length))
        if rc != 0:
            raise ValueError("Gauss-Newton matrix not positive definite")
        return dx, r.value, J.value, bool(lf.value)

    def grad(self, i: int, theta, l: float, goal):
        """Tip-distance cost |p_N - goal| at the equilibrium (theta, l) and its
        adjoint derivatives with respect to each actuator's pressure (per Pa),
        begin and end (per link unit).  Returns (cost, dP, dB, dE, status);
        status 1 = exact Hessian not positive definite (NaN derivatives)."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        na = int(self._keep["act_ptr"][i + 1] - self._keep["act_ptr"][i])
        dP, dB, dE = np.zeros(max(na, 1)), np.zeros(max(na, 1)), np.zeros(max(na, 1))
        c = C.c_double()
        rc = lib().orc_grad(C.byref(self.P), C.byref(self.B), self.T, int(i), th.size, _ptr(th), float(l),
                            float(goal[0]), float(goal[1]), C.byref(c), _ptr(dP), _ptr(dB), _ptr(dE))
        return c.value, dP[:na], dB[:na], dE[:na], rc

    def grad_path(self, i: int, theta, l: float, path):
        """Path cost (1/N) sum_k |p_k - q_k|^2 over the link end points p_1..p_N
        against targets path[k-1] = q_k ([N, 2], absolute), at the equilibrium
        (theta, l), and its adjoint derivatives as grad().  Returns
        (cost, dP, dB, dE, status)."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        q = np.asarray(path, dtype=np.float64).reshape(-1, 2)[: th.size]
        qx, qy = np.ascontiguousarray(q[:, 0]), np.ascontiguousarray(q[:, 1])
        na = int(self._keep["act_ptr"][i + 1] - self._keep["act_ptr"][i])
        dP, dB, dE = np.zeros(max(na, 1)), np.zeros(max(na, 1)), np.zeros(max(na, 1))
        c = C.c_double()
        rc = lib().orc_grad_path(C.byref(self.P), C.byref(self.B), self.T, int(i), th.size, _ptr(th), float(l),
                                 _ptr(qx), _ptr(qy), C.byref(c), _ptr(dP), _ptr(dB), _ptr(dE))
        return c.value, dP[:na], dB[:na], dE[:na], rc

    def poses(self, i: int, theta, l: float):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        N = th.size
        px, py, psi = np.zeros(N + 1), np.zeros(N + 1), np.zeros(N)
        lib().orc_poses(C.byref(self.P), C.byref(self.B), self.T, int(i), N, _ptr(th), float(l), _ptr(px),
                        _ptr(py), _ptr(psi))
        return px, py, psi

    def gaps(self, i: int, theta, l: float):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        N = th.size
        no = int(self._keep["obs_ptr"][i + 1] - self._keep["obs_ptr"][i])
        gap = np.zeros(max(N * no, 1))
        lib().orc_gaps(C.byref(self.P), C.byref(self.B), self.T, int(i), N, _ptr(th), float(l), _ptr(gap))
        return gap[: N * no].reshape(N, no)

    def sdf(self, o: int, x: float, y: float):
        nx, ny = C.c_double(), C.c_double()
        d = lib().orc_sdf(C.byref(self.B), int(o), float(x), float(y), C.byref(nx), C.byref(ny))
        return d, nx.value, ny.value

    def new_state(self):
        return dict(N=np.zeros(self.n, np.int32), theta=np.zeros(int(self.off[-1]) or 1),
                    l=np.zeros(self.n), iters=np.zeros(self.n, np.int32), resid=np.zeros(self.n),
                    status=np.zeros(self.n, np.int32), rls=np.zeros(self.n, np.int64),
                    conv=np.zeros(self.n, np.int32), evals=np.zeros(self.n, np.int64))

    def run(self, state: dict, n_steps: int, threads: int = 1) -> dict:
        """Grow every instance by up to n_steps links; state is updated in place."""
        s = state
        lib().orc_run(C.byref(self.P), C.byref(self.B), self.T, int(n_steps), _ptr(s["N"]), _ptr(s["theta"]),
                      _ptr(s["l"]), _ptr(s["iters"]), _ptr(s["resid"]), _ptr(s["status"]), _ptr(s["rls"]),
                      _ptr(s["conv"]), _ptr(s["evals"]), int(threads))
        return s

    def relax(self, state: dict, fix_length: bool = True, threads: int = 1) -> dict:
        """Re-solve every instance at its present links (no link added); the
        distal length held fixed with fix_length.  state is updated in place."""
        s = state
        lib().orc_relax(C.byref(self.P), C.byref(self.B), self.T, int(bool(fix_length)), _ptr(s["N"]),
                        _ptr(s["theta"]), _ptr(s["l"]), _ptr(s["iters"]), _ptr(s["resid"]), _ptr(s["status"]),
                        _ptr(s["rls"]), _ptr(s["conv"]), _ptr(s["evals"]), int(threads))
        return s

    def theta_of(self, state: dict, i: int):
        return state["theta"][self.off[i]: self.off[i] + state["N"][i]].copy()
