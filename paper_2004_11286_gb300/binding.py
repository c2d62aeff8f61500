"""Thin ctypes binding of ``include/lbm_mix.h``.

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch supplies device memory (population and scratch buffers), pinned host
buffers and the CUDA stream.  If the library is missing the constructor
raises; there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as ct
import os
from pathlib import Path
from typing import Optional

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "liblbm_mix.so"

PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
COUPLING = {"strong": 0, "weak": 1}
CLOSURE = {"exact": 0, "mlp": 1}
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_UNSUPPORTED", 3: "LBM_ERR_CUDA",
          4: "LBM_ERR_NONFINITE", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE"}

_DP = ct.POINTER(ct.c_double)


class lbm_mix_params(ct.Structure):
    _fields_ = [
        ("M", ct.c_int),
        ("molar_mass", _DP), ("cv_molar", _DP), ("D", _DP), ("mu", _DP), ("lambda_", _DP),
        ("omega_fixed", ct.c_double), ("omega1_fixed", ct.c_double), ("R_U", ct.c_double),
        ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("bc", ct.c_int * 6),
        ("slaved_species", ct.c_int), ("precision", ct.c_int), ("coupling", ct.c_int),
        ("closure", ct.c_int),
        ("fp64_cond_bound", ct.c_double),
        ("closure_residual_bound", ct.c_double),
        ("cv_poly", _DP), ("cv_terms", ct.c_int),
        ("jet_X", _DP), ("jet_u", ct.c_double * 2), ("jet_T", ct.c_double * 2), ("jet_P", ct.c_double * 2),
        ("jet_y0", ct.c_int), ("jet_y1", ct.c_int),
    ]


# Every function the header declares: name -> (restype, argtypes).
SIGNATURES = {
    "lbm_mix_create": (ct.c_int, [ct.POINTER(lbm_mix_params), ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "lbm_mix_required_bytes": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t)]),
    "lbm_mix_bind_buffers": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_size_t]),
    "lbm_mix_alloc_buffers": (ct.c_int, [ct.c_void_p]),
    "lbm_mix_init_fields": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "lbm_mix_step": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "lbm_mix_num_outputs": (ct.c_int, [ct.c_int]),
    "lbm_mix_get_moments": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int]),
    "lbm_mix_get_populations": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int]),
    "lbm_mix_set_populations": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int]),
    "lbm_mix_diagnostics": (ct.c_int, [ct.c_void_p, _DP]),
    "lbm_mix_synchronize": (ct.c_int, [ct.c_void_p]),
    "lbm_mix_set_reference": (ct.c_int, [ct.c_void_p, _DP, ct.c_double, ct.c_double]),
    "lbm_mix_halo_bytes": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_size_t)]),
    "lbm_mix_halo_pack": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p]),
    "lbm_mix_halo_unpack": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p]),
    "lbm_mix_step_count": (ct.c_longlong, [ct.c_void_p]),
    "lbm_mix_launch_count": (ct.c_longlong, [ct.c_void_p]),
    "lbm_mix_enable_kernel_timing": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "lbm_mix_kernel_times": (ct.c_int, [ct.c_void_p, _DP, ct.POINTER(ct.c_longlong), ct.c_int]),
    "lbm_mix_conserved_sums_noalloc": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int,
                                                  ct.c_void_p, ct.c_void_p]),
    "lbm_mix_closure_sizes": (ct.c_int, [ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                         ct.POINTER(ct.c_int)]),
    "lbm_mix_closure_set_weights": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int]),
    "lbm_mix_closure_get_weights": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int]),
    "lbm_mix_closure_samples": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "lbm_mix_closure_forward": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_longlong]),
    "lbm_mix_closure_loss_grad": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_longlong,
                                             ct.c_void_p, _DP]),
    "lbm_mix_closure_train": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_longlong, ct.c_int,
                                         ct.c_int, ct.c_double, _DP]),
    "lbm_mix_closure_stats": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong),
                                         ct.c_int]),
    "lbm_mix_batch_create": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "lbm_mix_batch_domain": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_void_p)]),
    "lbm_mix_batch_nodes": (ct.c_longlong, [ct.c_void_p]),
    "lbm_mix_batch_step": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "lbm_mix_batch_autotune": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int), _DP]),
    "lbm_mix_batch_set_config": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int]),
    "lbm_mix_batch_set_mode": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int]),
    "lbm_mix_batch_config": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int)]),
    "lbm_mix_batch_synchronize": (ct.c_int, [ct.c_void_p]),
    "lbm_mix_batch_destroy": (ct.c_int, [ct.c_void_p]),
    "lbm_mix_batch_last_error": (ct.c_char_p, [ct.c_void_p]),
    "lbm_mix_destroy": (ct.c_int, [ct.c_void_p]),
    "lbm_mix_last_error": (ct.c_char_p, [ct.c_void_p]),
}

_lib: Optional[ct.CDLL] = None


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load_library(path: Optional[os.PathLike] = None) -> ct.CDLL:
    """Load ``liblbm_mix.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path is not None else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is missing: build it with paper_2004_11286_gb300.build.build()")
    lib = ct.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(_DP)


def make_params(molar_mass, cv_molar, D, mu=None, lam=None, shape=(1, 1, 1), precision: str = "fp32",
                coupling: str = "strong", slaved: int = -1, omega_fixed: float = 0.0, omega1_fixed: float = 0.0,
                R_U: float = 1.0, fp64_cond_bound: float = 0.0, closure: str = "exact",
                closure_bound: float = 0.0, walls_x: bool = False, cv_poly=None, jets=None):
    """(lbm_mix_params, keepalive arrays) for one nz x ny x nx domain, periodic,
    or with bounce-back walls on both x faces (walls_x); cv_poly (M, K <= 3):
    temperature-dependent molar heats C-bar_{a,v}(T)/R_U = sum_k cv_poly[a, k] T^k.
    jets: the opposed-jets boundary set (LBM_BC_JET on the x faces,
    LBM_BC_OUTLET on the y faces); an object with y0, y1 (nozzle rows of the
    grid, frame included), X (2, M), u, T, P (2,)."""
    M = int(len(molar_mass))
    nz, ny, nx = (int(v) for v in shape)
    keep = [np.ascontiguousarray(np.asarray(v, dtype=np.float64).ravel()) for v in (molar_mass, cv_molar, D)]
    mu_a = None if mu is None else np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    lam_a = None if lam is None else np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
    keep += [mu_a, lam_a]
    p = lbm_mix_params()
    p.M = M
    p.molar_mass, p.cv_molar, p.D = (_dp(a) for a in keep[:3])
    p.mu = _dp(mu_a)
    p.lambda_ = _dp(lam_a)
    p.omega_fixed, p.omega1_fixed, p.R_U = float(omega_fixed), float(omega1_fixed), float(R_U)
    p.nx, p.ny, p.nz = nx, ny, nz
    for k in range(6):
        p.bc[k] = 1 if (walls_x and k < 2) else 0
    if jets is not None:
        for k in range(4):
            p.bc[k] = 2 if k < 2 else 3
        jx = np.ascontiguousarray(np.asarray(jets.X, dtype=np.float64).reshape(2, M))
        keep.append(jx)
        p.jet_X = _dp(jx)
        for k in range(2):
            p.jet_u[k], p.jet_T[k], p.jet_P[k] = float(jets.u[k]), float(jets.T[k]), float(jets.P[k])
        p.jet_y0, p.jet_y1 = int(jets.y0), int(jets.y1)
    else:
        p.jet_X = _dp(None)
    p.slaved_species = int(slaved)
    p.precision = PREC[precision]
    p.coupling = COUPLING[coupling]
    p.closure = CLOSURE[closure]
    p.fp64_cond_bound = float(fp64_cond_bound)
    p.closure_residual_bound = float(closure_bound)
    if cv_poly is not None:
        cp = np.ascontiguousarray(np.asarray(cv_poly, dtype=np.float64).reshape(M, -1))
        keep.append(cp)
        p.cv_poly = _dp(cp)
        p.cv_terms = int(cp.shape[1])
    else:
        p.cv_poly = _dp(None)
        p.cv_terms = 0
    return p, keep


class LbmMix:
    """One simulation handle: an nz x ny x nx grid of M species + f + g,
    periodic, or closed by bounce-back walls on both x faces (walls_x).

    Fields cross the boundary as float64 arrays: NumPy arrays are host
    pointers, torch CUDA tensors are device pointers.
    """

    def __init__(self, molar_mass, cv_molar, D, mu=None, lam=None, shape=(1, 1, 1),
                 precision: str = "fp32", coupling: str = "strong", slaved: int = -1,
                 omega_fixed: float = 0.0, omega1_fixed: float = 0.0, R_U: float = 1.0,
                 fp64_cond_bound: float = 0.0, closure: str = "exact", closure_bound: float = 0.0,
                 walls_x: bool = False, device=None, stream=None, cv_poly=None, jets=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.device = torch.device(device if device is not None else "cuda")
        self.M = int(len(molar_mass))
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        self.N = nx * ny * nz
        p, self._keep = make_params(molar_mass, cv_molar, D, mu=mu, lam=lam, shape=shape, precision=precision,
                                    coupling=coupling, slaved=slaved, omega_fixed=omega_fixed,
                                    omega1_fixed=omega1_fixed, R_U=R_U, fp64_cond_bound=fp64_cond_bound,
                                    closure=closure, closure_bound=closure_bound, walls_x=walls_x,
                                    cv_poly=cv_poly, jets=jets)
        self._owned = True
        self.precision = precision
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ct.c_void_p()
            st = self.lib.lbm_mix_create(ct.byref(p), ct.c_void_p(self.stream.cuda_stream), ct.byref(h))
            if st != 0:
                raise LbmError(st, self.lib.lbm_mix_last_error(None).decode())
            self.h = h
            pb, sb = ct.c_size_t(), ct.c_size_t()
            self._check(self.lib.lbm_mix_required_bytes(self.h, ct.byref(pb), ct.byref(sb)))
            self.pops_buf = torch.empty(pb.value, dtype=torch.uint8, device=self.device)
            self.scratch_buf = torch.empty(sb.value, dtype=torch.uint8, device=self.device)
            self._check(self.lib.lbm_mix_bind_buffers(self.h, ct.c_void_p(self.pops_buf.data_ptr()), pb.value,
                                                      ct.c_void_p(self.scratch_buf.data_ptr()), sb.value))

    # -- helpers -------------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            raise LbmError(st, self.lib.lbm_mix_last_error(self.h).decode())

    def _ptr(self, a, n_expected: int):
        """(pointer, host_flag, keepalive) for a float64 array of n elements."""
        torch = self._torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n_expected:
                raise ValueError("expected a contiguous float64 tensor of %d elements" % n_expected)
            if a.is_cuda:
                return ct.c_void_p(a.data_ptr()), 0, a
            return ct.c_void_p(a.data_ptr()), 1, a
        arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if arr.size != n_expected:
            raise ValueError("expected %d elements, got %d" % (n_expected, arr.size))
        return ct.c_void_p(arr.ctypes.data), 1, arr

    # -- API -----------------------------------------------------------------
    def init_fields(self, X, u, T, P):
        N, M = self.N, self.M
        px, hx, kx = self._ptr(X, M * N)
        pu, hu, ku = self._ptr(u, 3 * N)
        pt, ht, kt = self._ptr(T, N)
        pp, hp, kp = self._ptr(P, N)
        if len({hx, hu, ht, hp}) != 1:
            raise ValueError("X, u, T, P must all be host arrays or all device tensors")
        self._check(self.lib.lbm_mix_init_fields(self.h, px, pu, pt, pp, hx))

    def step(self, n: int = 1):
        self._check(self.lib.lbm_mix_step(self.h, int(n)))

    @property
    def n_outputs(self) -> int:
        return int(self.lib.lbm_mix_num_outputs(self.M))

    def moments(self, out=None):
        """Observables [6+5M][N] (float64): NumPy on the host unless ``out``
        is a device tensor."""
        n = self.n_outputs * self.N
        if out is None:
            out = np.empty(n, dtype=np.float64)
        p, host, keep = self._ptr(out, n)
        self._check(self.lib.lbm_mix_get_moments(self.h, p, host))
        return out

    def moments_dict(self):
        nz, ny, nx = self.shape
        M = self.M
        o = self.moments().reshape(self.n_outputs, nz, ny, nx)
        return dict(rho=o[0], u=o[1:4], T=o[4], P=o[5], X=o[6:6 + M], Y=o[6 + M:6 + 2 * M],
                    V=o[6 + 2 * M:].reshape(M, 3, nz, ny, nx))

    def populations(self, out=None):
        n = (self.M + 2) * 27 * self.N
        if out is None:
            out = np.empty(n, dtype=np.float64)
        p, host, keep = self._ptr(out, n)
        self._check(self.lib.lbm_mix_get_populations(self.h, p, host))
        if isinstance(out, np.ndarray):
            return out.reshape((self.M + 2, 27) + self.shape)
        return out

    def set_populations(self, pops):
        n = (self.M + 2) * 27 * self.N
        p, host, keep = self._ptr(pops, n)
        self._check(self.lib.lbm_mix_set_populations(self.h, p, host))

    def diagnostics(self):
        out = np.empty(self.M + 5, dtype=np.float64)
        self._check(self.lib.lbm_mix_diagnostics(self.h, out.ctypes.data_as(_DP)))
        return out

    def synchronize(self):
        self._check(self.lib.lbm_mix_synchronize(self.h))

    def set_reference(self, Y, T: float, rho: float):
        """Fix the reference rest state (mass fractions Y, temperature, density)."""
        y = np.ascontiguousarray(np.asarray(Y, dtype=np.float64))
        if y.size != self.M:
            raise ValueError("Y must have M entries")
        self._check(self.lib.lbm_mix_set_reference(self.h, y.ctypes.data_as(_DP), float(T), float(rho)))

    def halo_bytes(self, ghost: int) -> int:
        b = ct.c_size_t()
        self._check(self.lib.lbm_mix_halo_bytes(self.h, int(ghost), ct.byref(b)))
        return int(b.value)

    def halo_pack(self, face: int, ghost: int, buf):
        """Copy the `ghost` interior planes next to z face `face` into the
        device tensor `buf` (uint8, halo_bytes(ghost) bytes)."""
        self._check(self.lib.lbm_mix_halo_pack(self.h, int(face), int(ghost), ct.c_void_p(buf.data_ptr())))

    def halo_unpack(self, face: int, ghost: int, buf):
        """Copy the device tensor `buf` into the ghost planes of z face `face`."""
        self._check(self.lib.lbm_mix_halo_unpack(self.h, int(face), int(ghost), ct.c_void_p(buf.data_ptr())))

    KERNEL_NAMES = ("collide_stream", "grad_GK", "grad_X")

    def enable_kernel_timing(self, on: bool = True):
        self._check(self.lib.lbm_mix_enable_kernel_timing(self.h, int(bool(on))))

    def kernel_times(self):
        """{kernel: (total_ms, launches)} for the steps recorded since the last query."""
        ms = np.zeros(3)
        cnt = (ct.c_longlong * 3)()
        n = self.lib.lbm_mix_kernel_times(self.h, ms.ctypes.data_as(_DP), cnt, 3)
        if n < 0:
            raise LbmError(3, "kernel_times failed")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KERNEL_NAMES)}

    # -- learned closure -----------------------------------------------------
    def closure_sizes(self):
        """(F, O, number of packed FP32 weights) of this handle's network."""
        return closure_sizes(self.M)

    def _f32(self, t, n: int):
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and t.numel() == n):
            raise ValueError("expected a contiguous CUDA float32 tensor of %d elements" % n)
        return ct.c_void_p(t.data_ptr())

    def set_closure_weights(self, w):
        """FP32 master weights (packed; NumPy host array or CUDA tensor)."""
        torch = self._torch
        nw = self.closure_sizes()[2]
        if isinstance(w, torch.Tensor) and w.is_cuda:
            self._check(self.lib.lbm_mix_closure_set_weights(self.h, self._f32(w, nw), 0))
        else:
            a = np.ascontiguousarray(np.asarray(w, dtype=np.float32).ravel())
            if a.size != nw:
                raise ValueError("expected %d weights" % nw)
            self._check(self.lib.lbm_mix_closure_set_weights(self.h, ct.c_void_p(a.ctypes.data), 1))

    def closure_weights(self) -> np.ndarray:
        w = np.empty(self.closure_sizes()[2], dtype=np.float32)
        self._check(self.lib.lbm_mix_closure_get_weights(self.h, ct.c_void_p(w.ctypes.data), 1))
        return w

    def closure_samples(self):
        """(features [N, F], exact normalised targets [N, O]) as CUDA float32 tensors."""
        torch = self._torch
        F, O, _ = self.closure_sizes()
        feat = torch.empty((self.N, F), dtype=torch.float32, device=self.device)
        tgt = torch.empty((self.N, O), dtype=torch.float32, device=self.device)
        self._check(self.lib.lbm_mix_closure_samples(self.h, ct.c_void_p(feat.data_ptr()),
                                                     ct.c_void_p(tgt.data_ptr())))
        return feat, tgt

    def closure_forward(self, feat):
        """Tensor-core network outputs [n, O] for CUDA float32 features [n, F]."""
        torch = self._torch
        F, O, _ = self.closure_sizes()
        n = feat.shape[0]
        out = torch.empty((n, O), dtype=torch.float32, device=self.device)
        self._check(self.lib.lbm_mix_closure_forward(self.h, self._f32(feat, n * F),
                                                     ct.c_void_p(out.data_ptr()), n))
        return out

    def closure_loss_grad(self, feat, tgt):
        """(loss, gradient [n_weights] CUDA float32) from the FP32 training kernels."""
        torch = self._torch
        F, O, nw = self.closure_sizes()
        n = feat.shape[0]
        g = torch.empty(nw, dtype=torch.float32, device=self.device)
        loss = ct.c_double()
        self._check(self.lib.lbm_mix_closure_loss_grad(self.h, self._f32(feat, n * F), self._f32(tgt, n * O), n,
                                                       ct.c_void_p(g.data_ptr()), ct.byref(loss)))
        return loss.value, g

    def closure_train(self, feat, tgt, batch: int, steps: int, lr: float) -> float:
        """Adam steps on the (already shuffled) pairs; returns the last mini-batch loss."""
        F, O, _ = self.closure_sizes()
        n = feat.shape[0]
        loss = ct.c_double()
        self._check(self.lib.lbm_mix_closure_train(self.h, self._f32(feat, n * F), self._f32(tgt, n * O), n,
                                                   int(batch), int(steps), float(lr), ct.byref(loss)))
        return loss.value

    def closure_stats(self, reset: bool = False):
        """(accepted, fallback) node counts of the network closure."""
        a, f = ct.c_longlong(), ct.c_longlong()
        self._check(self.lib.lbm_mix_closure_stats(self.h, ct.byref(a), ct.byref(f), int(bool(reset))))
        return a.value, f.value

    @property
    def step_count(self) -> int:
        return int(self.lib.lbm_mix_step_count(self.h))

    @property
    def launch_count(self) -> int:
        return int(self.lib.lbm_mix_launch_count(self.h))

    @classmethod
    def _borrowed(cls, lib, h, M, shape, precision, device, stream):
        """Wrapper of a handle owned by a batch (never destroyed here)."""
        import torch
        self = cls.__new__(cls)
        self._torch, self.lib, self.h = torch, lib, h
        self.M, self.shape = int(M), tuple(int(v) for v in shape)
        self.N = int(np.prod(self.shape))
        self.precision, self.device, self.stream = precision, device, stream
        self._owned = False
        return self

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            self.lib.lbm_mix_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LbmBatch:
    """An ensemble of independent periodic domains stepped together.

    ``domains`` is a list of keyword dicts for :func:`make_params` (each with
    its own constants and shape; all share M, precision and coupling).
    ``self.domain(d)`` gives an :class:`LbmMix` view of domain d for
    init_fields, moments, populations and diagnostics."""

    def __init__(self, domains, device=None, stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.device = torch.device(device if device is not None else "cuda")
        nd = len(domains)
        arr = (lbm_mix_params * nd)()
        self._keep = []
        self._meta = []
        for d, kw in enumerate(domains):
            p, keep = make_params(**kw)
            arr[d] = p
            self._keep.append(keep)
            self._meta.append((len(kw["molar_mass"]), tuple(kw["shape"]), kw.get("precision", "fp32")))
        self._params = arr
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            b = ct.c_void_p()
            st = self.lib.lbm_mix_batch_create(ct.cast(arr, ct.c_void_p), nd, ct.c_void_p(self.stream.cuda_stream),
                                               ct.byref(b))
            if st != 0:
                raise LbmError(st, self.lib.lbm_mix_last_error(None).decode())
        self.b = b
        self.nd = nd
        self._views = []
        for d in range(nd):
            h = ct.c_void_p()
            self._check(self.lib.lbm_mix_batch_domain(self.b, d, ct.byref(h)))
            M, shape, prec = self._meta[d]
            self._views.append(LbmMix._borrowed(self.lib, h, M, shape, prec, self.device, self.stream))

    def _check(self, st: int):
        if st != 0:
            raise LbmError(st, self.lib.lbm_mix_batch_last_error(self.b).decode())

    def domain(self, d: int) -> LbmMix:
        return self._views[d]

    @property
    def nodes(self) -> int:
        return int(self.lib.lbm_mix_batch_nodes(self.b))

    def step(self, n: int = 1):
        self._check(self.lib.lbm_mix_batch_step(self.b, int(n)))

    def autotune(self, trial_steps: int = 4):
        cfg = (ct.c_int * 5)()
        ms = ct.c_double()
        self._check(self.lib.lbm_mix_batch_autotune(self.b, int(trial_steps), cfg, ct.byref(ms)))
        return dict(grid_collide=cfg[0], block_stencil=cfg[1], grid_stencil=cfg[2], mode=cfg[3], branches=cfg[4],
                    ms_per_step=ms.value)

    def set_mode(self, mode: int, branches: int = 8):
        self._check(self.lib.lbm_mix_batch_set_mode(self.b, int(mode), int(branches)))

    def set_config(self, grid_collide: int, block_stencil: int, grid_stencil: int, use_graph: bool = True):
        self._check(self.lib.lbm_mix_batch_set_config(self.b, int(grid_collide), int(block_stencil),
                                                      int(grid_stencil), int(bool(use_graph))))

    def config(self):
        c = (ct.c_int * 10)()
        self._check(self.lib.lbm_mix_batch_config(self.b, c))
        keys = ("grid_collide", "block_stencil", "grid_stencil", "use_graph", "tiles_collide", "tiles_128",
                "tiles_256", "collide_block", "mode", "branches")
        return dict(zip(keys, list(c)))

    def synchronize(self):
        self._check(self.lib.lbm_mix_batch_synchronize(self.b))

    def close(self):
        if getattr(self, "b", None):
            for v in self._views:
                v.h = None
            self.lib.lbm_mix_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workload_params(wl, precision: str = "fp32", **kw):
    """make_params keywords for a ``workloads.Workload``."""
    params = wl.params()
    return dict(molar_mass=params["molar_mass"], cv_molar=params["cv_molar"], D=params["D"], mu=params["mu"],
                lam=params["lam"], shape=wl.shape, precision=precision, R_U=params["R_U"], **kw)


def closure_sizes(M: int):
    """(F, O, packed weight count) of the closure network for M species."""
    lib = load_library()
    F, O, nw = ct.c_int(), ct.c_int(), ct.c_int()
    rc = lib.lbm_mix_closure_sizes(int(M), ct.byref(F), ct.byref(O), ct.byref(nw))
    if rc != 0:
        raise LbmError(rc, lib.lbm_mix_last_error(None).decode())
    return F.value, O.value, nw.value


def conserved_sums_noalloc(pops, M: int, shape, sums, stream=None):
    """Conservation sums of device populations [M+2][27][N] into the device
    tensor ``sums`` [M+5] without any allocation (static scratch in the
    library).  Both tensors are CUDA float64 and contiguous."""
    import torch
    lib = load_library()
    nz, ny, nx = shape
    for t in (pops, sums):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("pops and sums must be contiguous CUDA float64 tensors")
    st = stream if stream is not None else torch.cuda.current_stream(pops.device)
    rc = lib.lbm_mix_conserved_sums_noalloc(ct.c_void_p(pops.data_ptr()), int(M), int(nx), int(ny), int(nz),
                                            ct.c_void_p(sums.data_ptr()), ct.c_void_p(st.cuda_stream))
    if rc != 0:
        raise LbmError(rc, lib.lbm_mix_last_error(None).decode())


def from_workload(wl, precision: str = "fp32", **kw) -> LbmMix:
    """Handle for a ``workloads.Workload`` (periodic grid, its species constants)."""
    params = wl.params()
    return LbmMix(params["molar_mass"], params["cv_molar"], params["D"], mu=params["mu"],
                  lam=params["lam"], shape=wl.shape, precision=precision, R_U=params["R_U"], **kw)
