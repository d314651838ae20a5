"""Python face of the dlma C ABI: one ``Context`` per lattice / device / stream.

Arrays are numpy complex128 (host memory, DLMA_MEM_HOST) or torch complex128
CUDA tensors (device memory, DLMA_MEM_DEVICE), in the canonical layouts of
include/dlma.h.  Outputs are allocated in the same kind of memory as the
inputs.  The methods only marshal arguments; every step runs in libdlma.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be a C-contiguous numpy array")
    return C.c_void_p(a.ctypes.data)


def _mem(a) -> int:
    return L.MEM_DEVICE if _is_torch(a) else L.MEM_HOST


def _empty_like(a, shape, dtype="complex"):
    if _is_torch(a):
        import torch
        dt = torch.complex128 if dtype == "complex" else torch.float64
        return torch.empty(shape, dtype=dt, device=a.device)
    return np.empty(shape, dtype=np.complex128 if dtype == "complex" else np.float64)


def _check_c128(a, shape, name):
    if _is_torch(a):
        import torch
        ok = a.dtype == torch.complex128 and a.is_cuda
    else:
        ok = isinstance(a, np.ndarray) and a.dtype == np.complex128
    if not ok:
        raise TypeError(f"{name} must be complex128 (numpy, or a CUDA torch tensor)")
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(a.shape)}, expected {tuple(shape)}")


class Context:
    """dlma_create / dlma_destroy around one L^3 x T lattice."""

    def __init__(self, L_: int, T: int, bc_t: int = 0, device: int = 0, stream=None):
        self.lib = L.load()
        self.L, self.T, self.bc_t = L_, T, bc_t
        self.V = L_ ** 3 * T
        self.Vs = L_ ** 3
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = None
        self.params = None          # (m0, c_sw) last set on the context
        lat = L.Lattice(L_, T, bc_t)
        h = C.c_void_p()
        st = self.lib.dlma_create(C.byref(lat), device, C.c_void_p(stream) if stream else None, C.byref(h))
        if st != L.DLMA_OK:
            raise L.DlmaError(st, "dlma_create failed")
        self.h = h

    # ------------------------------------------------------------------
    def _check(self, st, allow=()):
        if st != L.DLMA_OK and st not in allow:
            raise L.DlmaError(st, self.lib.dlma_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.dlma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------
    def dlma_set_memory_cap(self, nbytes: int):
        self._check(self.lib.dlma_set_memory_cap(self.h, int(nbytes)))

    def dlma_release_workspace(self):
        self._check(self.lib.dlma_release_workspace(self.h))

    def dlma_set_gauge(self, U):
        _check_c128(U, (self.V, 4, 3, 3), "links")
        self.params = None
        self._check(self.lib.dlma_set_gauge(self.h, _ptr(U), _mem(U)))

    def dlma_set_params(self, m0: float, c_sw: float):
        self._check(self.lib.dlma_set_params(self.h, float(m0), float(c_sw)))
        self.params = (float(m0), float(c_sw))

    def dlma_apply_Dw(self, psi, prec: int = L.FP64):
        n = psi.shape[0]
        _check_c128(psi, (n, self.V, 4, 3), "psi")
        out = _empty_like(psi, psi.shape)
        self._check(self.lib.dlma_apply_Dw(self.h, _ptr(psi), _ptr(out), n, prec, _mem(psi)))
        return out

    def dlma_apply_schur(self, psi_e, dagger: int = 0, prec: int = L.FP64):
        n = psi_e.shape[0]
        _check_c128(psi_e, (n, self.V // 2, 4, 3), "psi_e")
        out = _empty_like(psi_e, psi_e.shape)
        self._check(self.lib.dlma_apply_schur(self.h, _ptr(psi_e), _ptr(out), n, int(dagger), prec, _mem(psi_e)))
        return out

    def dlma_set_solver(self, solver: int):
        """L.SOLVER_BICGSTAB (default) or L.SOLVER_CGNE for the FP32 inner solves."""
        self._check(self.lib.dlma_set_solver(self.h, int(solver)))

    def dlma_solve(self, b, tol: float, inner: int = L.FP64, allow_not_converged: bool = False):
        n = b.shape[0]
        _check_c128(b, (n, self.V, 4, 3), "b")
        x = _empty_like(b, b.shape)
        info = (L.SolveInfo * n)()
        st = self.lib.dlma_solve(self.h, _ptr(b), _ptr(x), n, float(tol), inner, info, _mem(b))
        self._check(st, allow=(L.DLMA_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return x, [dict(iters_inner=i.iters_inner, iters_outer=i.iters_outer, true_resid=i.true_resid,
                        converged=bool(i.converged)) for i in info]

    def dlma_solve_adjoint(self, g, tol: float, inner: int = L.FP64):
        n = g.shape[0]
        _check_c128(g, (n, self.V, 4, 3), "g")
        y = _empty_like(g, g.shape)
        info = (L.SolveInfo * n)()
        self._check(self.lib.dlma_solve_adjoint(self.h, _ptr(g), _ptr(y), n, float(tol), inner, info, _mem(g)))
        return y

    def dlma_real_dot(self, a, b) -> float:
        if tuple(a.shape) != tuple(b.shape):
            raise ValueError("shape mismatch")
        n = 1
        for s in a.shape:
            n *= int(s)
        out = C.c_double()
        self._check(self.lib.dlma_real_dot(self.h, _ptr(a), _ptr(b), n, C.byref(out), _mem(a)))
        return out.value

    def dlma_set_checkpoint(self, on: bool):
        self._check(self.lib.dlma_set_checkpoint(self.h, 1 if on else 0))

    def dlma_correlators_backward(self, t_src: int, N: int, n_noise: int, w, tol: float, inner: int = L.FP32):
        """(dL/dm0, dL/deta) of L = sum_t w(t) Re C_PS(t) for the last checkpointed forward."""
        if _is_torch(w):
            import torch
            w = w.detach().to(torch.float64).contiguous()
            deta = torch.empty((n_noise, self.Vs, 4, 3), dtype=torch.complex128, device=w.device)
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            deta = np.empty((n_noise, self.Vs, 4, 3), dtype=np.complex128)
        dm0 = C.c_double()
        self._check(self.lib.dlma_correlators_backward(self.h, int(t_src), int(N), int(n_noise), _ptr(w),
                                                       float(tol), inner, C.byref(dm0), _ptr(deta), None, _mem(w)))
        return dm0.value, deta

    def dlma_apply_laplacian(self, v):
        n = v.shape[0]
        _check_c128(v, (n, self.V, 3), "v")
        out = _empty_like(v, v.shape)
        self._check(self.lib.dlma_apply_laplacian(self.h, _ptr(v), _ptr(out), n, _mem(v)))
        return out

    def dlma_laplacian_eigs(self, t: int, N: int, tol: float = 1e-10, device_out: bool = False, want_vecs=True):
        nt = self.T if t < 0 else 1
        evals = np.empty((nt, N), dtype=np.float64)
        evecs = None
        mem = L.MEM_HOST
        if want_vecs:
            if device_out:
                import torch
                evecs = torch.empty((nt, N, self.Vs, 3), dtype=torch.complex128, device="cuda")
                mem = L.MEM_DEVICE
            else:
                evecs = np.empty((nt, N, self.Vs, 3), dtype=np.complex128)
        self._check(self.lib.dlma_laplacian_eigs(self.h, int(t), int(N), float(tol), _ptr(evals), _ptr(evecs), mem))
        if t >= 0:
            return evals[0], (evecs[0] if evecs is not None else None)
        return evals, evecs

    def dlma_make_sources(self, t_src: int, V, eta):
        N = V.shape[0]
        nn = eta.shape[0]
        _check_c128(V, (N, self.Vs, 3), "V")
        _check_c128(eta, (nn, self.Vs, 4, 3), "eta")
        b = _empty_like(V, (4 * N + 5 * nn, self.V, 4, 3))
        self._check(self.lib.dlma_make_sources(self.h, int(t_src), N, _ptr(V), nn, _ptr(eta), _ptr(b), _mem(V)))
        return b

    def dlma_project(self, t: int, V, psi):
        N = V.shape[-3]
        nt = self.T if t < 0 else 1
        _check_c128(V, ((self.T,) if t < 0 else ()) + (N, self.Vs, 3), "V")
        n = psi.shape[0]
        _check_c128(psi, (n, self.V, 4, 3), "psi")
        coeff = _empty_like(psi, (n, nt, 4, N))
        self._check(self.lib.dlma_project(self.h, int(t), _ptr(V), N, _ptr(psi), n, _ptr(coeff), _mem(psi)))
        return coeff

    @staticmethod
    def _parts(out):
        """The five correlator arrays of dlma_contract / dlma_correlators, as the library wrote them."""
        return dict(zip(("C_dist", "C_rest", "C_mixed", "C_mixed_src", "C"), out))

    @staticmethod
    def _infos(info):
        return [dict(iters_inner=i.iters_inner, iters_outer=i.iters_outer, true_resid=i.true_resid,
                     converged=bool(i.converged)) for i in info]

    def dlma_contract(self, t_src: int, V, phi, n_noise: int):
        N = V.shape[1]
        _check_c128(V, (self.T, N, self.Vs, 3), "V")
        _check_c128(phi, (4 * N + 5 * n_noise, self.V, 4, 3), "phi")
        out = [np.empty((4, self.T), dtype=np.complex128) for _ in range(5)]
        self._check(self.lib.dlma_contract(self.h, int(t_src), N, _ptr(V), int(n_noise), _ptr(phi),
                                           *[_ptr(o) for o in out], _mem(phi)))
        return self._parts(out)

    def dlma_correlators(self, t_src: int, N: int, eta, tol: float, inner: int = L.FP32):
        """C_dist, C_rest, C_mixed, C_mixed_src and the Eq. 2 total C (all from the library)."""
        nn = eta.shape[0]
        _check_c128(eta, (nn, self.Vs, 4, 3), "eta")
        out = [np.empty((4, self.T), dtype=np.complex128) for _ in range(5)]
        info = (L.SolveInfo * (4 * N + 5 * nn))()
        self._check(self.lib.dlma_correlators(self.h, int(t_src), int(N), nn, _ptr(eta), float(tol), inner,
                                              *[_ptr(o) for o in out], info, _mem(eta)))
        res = self._parts(out)
        res["info"] = self._infos(info)
        return res

    def dlma_correlators_diluted(self, t_src: int, N: int, eta, tol: float, inner: int = L.FP32):
        """Colour x even-odd diluted wall sources, spin-explicit; eta complex [n_noise, L^3, 3]."""
        nn = eta.shape[0]
        _check_c128(eta, (nn, self.Vs, 3), "eta")
        out = [np.empty((4, self.T), dtype=np.complex128) for _ in range(5)]
        info = (L.SolveInfo * (4 * N + 48 * nn))()
        self._check(self.lib.dlma_correlators_diluted(self.h, int(t_src), int(N), nn, _ptr(eta), float(tol), inner,
                                                      *[_ptr(o) for o in out], info, _mem(eta)))
        res = self._parts(out)
        res["info"] = self._infos(info)
        return res

    def dlma_correlators_plain(self, t_src: int, eta, tol: float, inner: int = L.FP32):
        """The plain stochastic estimator (no distillation): eta complex [n_noise, L^3, 4, 3]
        (undiluted) or [n_noise, L^3, 3] (colour x even-odd diluted wall sources)."""
        nn = eta.shape[0]
        diluted = len(eta.shape) == 3
        _check_c128(eta, (nn, self.Vs, 3) if diluted else (nn, self.Vs, 4, 3), "eta")
        out = np.empty((4, self.T), dtype=np.complex128)
        info = (L.SolveInfo * ((24 if diluted else 4) * nn))()
        self._check(self.lib.dlma_correlators_plain(self.h, int(t_src), nn, _ptr(eta), int(diluted), float(tol),
                                                    inner, _ptr(out), info, _mem(eta)))
        return {"C": out, "info": self._infos(info)}

    def dlma_dirac_eigs(self, N: int, tol: float = 1e-10, device_out: bool = False):
        """(lambda [N], u [N, V/2, 4, 3]) of Qhat = g5 Dhat with the smallest |lambda|."""
        evals = np.empty(N, dtype=np.float64)
        if device_out:
            import torch
            evecs = torch.empty((N, self.V // 2, 4, 3), dtype=torch.complex128, device="cuda")
        else:
            evecs = np.empty((N, self.V // 2, 4, 3), dtype=np.complex128)
        self._check(self.lib.dlma_dirac_eigs(self.h, int(N), float(tol), _ptr(evals), _ptr(evecs), _mem(evecs)))
        return evals, evecs

    def dlma_dirac_project(self, v, conj_g5: bool = False):
        """P v (or g5 P g5 v) over the cached Dirac low modes; v complex [n, V/2, 4, 3]."""
        n = v.shape[0]
        _check_c128(v, (n, self.V // 2, 4, 3), "v")
        out = _empty_like(v, v.shape)
        self._check(self.lib.dlma_dirac_project(self.h, _ptr(v), _ptr(out), n, int(bool(conj_g5)), _mem(v)))
        return out

    def dlma_index_tables(self):
        eo = np.empty(self.V, dtype=np.int32)
        nbr = np.empty((2, 8, self.V // 2), dtype=np.int32)
        self._check(self.lib.dlma_index_tables(self.h, _ptr(eo), _ptr(nbr)))
        return eo, nbr

    def dlma_kernel_launches(self) -> int:
        return int(self.lib.dlma_kernel_launches(self.h))

    def dlma_last_timing(self):
        """The eight timing slots of the last call (meaning per call in include/dlma.h)."""
        out = np.zeros(8, dtype=np.float64)
        self._check(self.lib.dlma_last_timing(self.h, _ptr(out), 8))
        return out

    def dlma_checkpoint_serial(self) -> int:
        return int(self.lib.dlma_checkpoint_serial(self.h))
