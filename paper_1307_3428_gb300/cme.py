"""Python binding of the CME C ABI (include/cme.h): argument marshalling only.

Every step of the integration runs in the CUDA library `_lib/libcme.so`; this module converts
numpy arrays and torch tensors to plain pointers.  There is no CPU fallback: if the library is
missing, `load()` raises.

PyTorch supplies device memory (through the library's allocator hooks, backed by the torch
caching allocator) and streams (`torch.cuda.Stream`).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcme.so")

CME_OK = 0
ERRORS = {
    -1: "CME_ERR_INVALID_ARG",
    -2: "CME_ERR_UNSUPPORTED_N",
    -3: "CME_ERR_CUDA",
    -4: "CME_ERR_NONFINITE",
    -5: "CME_ERR_TIMEOUT",
    -6: "CME_ERR_OOM",
    -7: "CME_ERR_STATE",
}
FP64, FP32 = 0, 1
RK4IP, STRANG = 0, 1
POWER, FIELD_D, FIELD_EQ1 = 0, 1, 2
HOST, DEVICE = 0, 1


class CmeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("integrator", ctypes.c_int),
                ("radix", ctypes.c_int), ("inst_per_cta", ctypes.c_int),
                ("steps_per_launch", ctypes.c_long), ("use_graph", ctypes.c_int),
                ("persistent", ctypes.c_int), ("cluster", ctypes.c_int)]


class Grads(ctypes.Structure):
    _fields_ = [(n, ctypes.POINTER(ctypes.c_double)) for n in
                ("loss", "d_sigma", "d_A_in", "d_D2", "d_D3", "d_omega", "d_kappa", "d_D0")] + \
               [("stored", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None

# (name, restype, argtypes) for every entry point of include/cme.h
_VP, _DP, _IP = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
_SIGS = [
    ("cme_default_options", None, [ctypes.POINTER(Options)]),
    ("cme_create", ctypes.c_int, [ctypes.c_int, _DP, _DP, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(_VP)]),
    ("cme_create_eq2", ctypes.c_int, [ctypes.c_int, _DP, _DP, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(_VP)]),
    ("cme_set_field", ctypes.c_int, [_VP, _DP]),
    ("cme_set_modes", ctypes.c_int, [_VP, ctypes.c_int]),
    ("cme_set_kerr", ctypes.c_int, [_VP, _DP]),
    ("cme_destroy", None, [_VP]),
    ("cme_batch_create", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int,
                                        ctypes.POINTER(Options), _VP, ctypes.POINTER(_VP)]),
    ("cme_batch_destroy", None, [_VP]),
    ("cme_batch_info", ctypes.c_int, [_VP, _IP, ctypes.POINTER(ctypes.c_long), _IP, _IP]),
    ("cme_batch_stream", _VP, [_VP]),
    ("cme_batch_plan", ctypes.c_int, [_VP, ctypes.c_int, _IP, _IP, _IP, _IP, _IP]),
    ("cme_step", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_long]),
    ("cme_synchronize", ctypes.c_int, [_VP]),
    ("cme_autotune", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_long, ctypes.POINTER(Options)]),
    ("cme_spectrum", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _DP]),
    ("cme_get_state", ctypes.c_int, [_VP, _DP, ctypes.c_int]),
    ("cme_set_state", ctypes.c_int, [_VP, _DP, ctypes.c_int]),
    ("cme_checkpoint_size", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    ("cme_checkpoint_save", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("cme_checkpoint_load", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("cme_get_time", ctypes.c_int, [_VP, _DP]),
    ("cme_set_time", ctypes.c_int, [_VP, ctypes.c_double]),
    ("cme_status", ctypes.c_int, [_VP, _IP]),
    ("cme_debug_fault", ctypes.c_int, [_VP, ctypes.c_int]),
    ("cme_grad", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_long, _DP, ctypes.c_double,
                                ctypes.c_long, ctypes.POINTER(Grads)]),
    ("cme_set_grad_memory", ctypes.c_int, [_VP, ctypes.c_longlong]),
    ("cme_rk4ip_noalloc", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_long, _VP, _VP, _VP, _VP, _VP]),
    ("cme_transform", ctypes.c_int, [_VP, ctypes.c_int, _DP, ctypes.c_int]),
    ("cme_eval_rhs", ctypes.c_int, [_VP, _DP, ctypes.c_int]),
    ("cme_set_allocator", ctypes.c_int, [ALLOC_FN, FREE_FN, _VP]),
    ("cme_fma_peak", ctypes.c_int, [ctypes.c_int, _DP]),
    ("cme_l2_peak", ctypes.c_int, [ctypes.c_size_t, _DP]),
    ("cme_kernel_launches", ctypes.c_long, []),
    ("cme_last_error", ctypes.c_char_p, []),
    ("cme_version", ctypes.c_char_p, []),
]


def load() -> ctypes.CDLL:
    """Load libcme.so (built by `__graft_entry__.build()`); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CME CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_names():
    return [s[0] for s in _SIGS]


def _check(rc: int):
    if rc != CME_OK:
        raise CmeError(rc, load().cme_last_error().decode(errors="replace"))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _interleave(z) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    return np.ascontiguousarray(z.view(np.float64))


# ---- torch-backed device memory --------------------------------------------------------------
_torch_hooks = None


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_hooks
    import torch

    live = {}

    def _alloc(nbytes, ctx):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(ptr, ctx):
        live.pop(ptr, None)

    _torch_hooks = (ALLOC_FN(_alloc), FREE_FN(_free), live)
    _check(load().cme_set_allocator(_torch_hooks[0], _torch_hooks[1], None))


class Instance:
    """Host-side parameters of one CME problem (see cme_create)."""

    def __init__(self, N, kappa, omega, g0, kappa_ext, A_in, sigma, D0=None, M=None,
                 g0_mu=None):
        lib = load()
        kap = np.ascontiguousarray(kappa, dtype=np.float64)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        h = ctypes.c_void_p()
        A_in = complex(A_in)
        _check(lib.cme_create(int(N), _dptr(kap), _dptr(om), float(g0), float(kappa_ext),
                              A_in.real, A_in.imag, float(sigma), ctypes.byref(h)))
        self.handle = h
        self.N = int(N)
        if D0 is not None:
            self.set_field(D0)
        if M is not None:
            self.set_modes(M)
        if g0_mu is not None:
            self.set_kerr(g0_mu)

    @classmethod
    def from_eq2(cls, N, Omega, f0, kappa_rel=None, D0=None, M=None) -> "Instance":
        """An instance of the normalised Eq. 2 (cme_create_eq2)."""
        self = cls.__new__(cls)
        om = np.ascontiguousarray(Omega, dtype=np.float64)
        kr = None if kappa_rel is None else np.ascontiguousarray(kappa_rel, dtype=np.float64)
        h = ctypes.c_void_p()
        f0 = complex(f0)
        _check(load().cme_create_eq2(int(N), None if kr is None else _dptr(kr), _dptr(om),
                                     f0.real, f0.imag, ctypes.byref(h)))
        self.handle = h
        self.N = int(N)
        if D0 is not None:
            self.set_field(D0)
        if M is not None:
            self.set_modes(M)
        return self

    @classmethod
    def from_workload(cls, inst) -> "Instance":
        return cls(inst.N, inst.kappa, inst.omega, inst.g0, inst.kappa_ext, inst.A_in,
                   inst.sigma, inst.D0, getattr(inst, "M", None), getattr(inst, "g0_mu", None))

    def set_modes(self, M: int):
        """Physical mode count (cme_set_modes): the centred M of the N modes."""
        _check(load().cme_set_modes(self.handle, int(M)))

    def set_kerr(self, g0_mu):
        """Per-mode Kerr coefficients g0_mu (cme_set_kerr; centred); None restores g0."""
        if g0_mu is None:
            _check(load().cme_set_kerr(self.handle, None))
        else:
            g = np.ascontiguousarray(g0_mu, dtype=np.float64)
            assert g.size == self.N
            _check(load().cme_set_kerr(self.handle, _dptr(g)))

    def set_field(self, D0):
        d = _interleave(D0)
        _check(load().cme_set_field(self.handle, _dptr(d)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.cme_destroy(self.handle)
            self.handle = None


class Batch:
    """Device-resident batch of instances (see cme_batch_create)."""

    def __init__(self, instances: Sequence, precision=FP64, integrator=RK4IP, radix=0,
                 inst_per_cta=0, steps_per_launch=0, use_graph=False, stream=None,
                 persistent=0, cluster=0):
        lib = load()
        insts = [i if isinstance(i, Instance) else Instance.from_workload(i) for i in instances]
        opt = Options()
        lib.cme_default_options(ctypes.byref(opt))
        opt.precision, opt.integrator = int(precision), int(integrator)
        opt.radix, opt.inst_per_cta = int(radix), int(inst_per_cta)
        opt.steps_per_launch, opt.use_graph = int(steps_per_launch), int(bool(use_graph))
        opt.persistent = int(persistent)
        opt.cluster = int(cluster)
        arr = (ctypes.c_void_p * len(insts))(*[i.handle.value for i in insts])
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if stream else None
        _check(lib.cme_batch_create(arr, len(insts), ctypes.byref(opt), s, ctypes.byref(h)))
        self.handle = h
        self.sizes = [i.N for i in insts]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.total = int(self.offsets[-1])
        self.count = len(insts)
        self.last_grad_schedule = None   # "stored" or "checkpoint" after a grad call
        self.precision = precision
        self.integrator = integrator

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.cme_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    @property
    def stream(self) -> int:
        return load().cme_batch_stream(self.handle) or 0

    def step(self, h: float, nsteps: int):
        _check(load().cme_step(self.handle, float(h), int(nsteps)))

    def synchronize(self):
        _check(load().cme_synchronize(self.handle))

    def plan(self, group: int = 0) -> dict:
        """The launch plan of one launch group (cme_batch_plan)."""
        v = [ctypes.c_int() for _ in range(5)]
        _check(load().cme_batch_plan(self.handle, int(group), *[ctypes.byref(x) for x in v]))
        return dict(zip(("N", "radix", "inst_per_cta", "cluster", "persistent"),
                        (x.value for x in v)))

    def autotune(self, h: float, probe_steps: int = 200) -> dict:
        opt = Options()
        _check(load().cme_autotune(self.handle, float(h), int(probe_steps), ctypes.byref(opt)))
        return {f: getattr(opt, f) for f, _ in Options._fields_}

    def split(self, flat: np.ndarray):
        return [flat[self.offsets[i]:self.offsets[i + 1]] for i in range(self.count)]

    def spectrum(self, what=POWER, idx: int = -1) -> np.ndarray:
        n = self.total if idx < 0 else self.sizes[idx]
        if what == POWER:
            out = np.empty(n, dtype=np.float64)
        else:
            out = np.empty(2 * n, dtype=np.float64)
        _check(load().cme_spectrum(self.handle, int(idx), int(what), _dptr(out)))
        return out if what == POWER else out.view(np.complex128)

    def get_state(self) -> np.ndarray:
        out = np.empty(2 * self.total, dtype=np.float64)
        _check(load().cme_get_state(self.handle, _dptr(out), HOST))
        return out.view(np.complex128)

    def set_state(self, D):
        d = _interleave(D)
        assert d.size == 2 * self.total
        _check(load().cme_set_state(self.handle, _dptr(d), HOST))

    def get_state_device(self, ptr: int):
        _check(load().cme_get_state(self.handle, ctypes.cast(ctypes.c_void_p(ptr), _DP), DEVICE))

    def set_state_device(self, ptr: int):
        _check(load().cme_set_state(self.handle, ctypes.cast(ctypes.c_void_p(ptr), _DP), DEVICE))

    def time(self) -> float:
        t = ctypes.c_double()
        _check(load().cme_get_time(self.handle, ctypes.byref(t)))
        return t.value

    def set_time(self, tau: float):
        _check(load().cme_set_time(self.handle, float(tau)))

    def status(self) -> np.ndarray:
        out = np.zeros(self.count, dtype=np.int32)
        _check(load().cme_status(self.handle, out.ctypes.data_as(_IP)))
        return out

    def debug_fault(self, what: int):
        """Test of the bounded device waits (cme_debug_fault): 1 makes later cluster
        all-to-alls run out their waits, 0 restores normal operation."""
        _check(load().cme_debug_fault(self.handle, int(what)))

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t()
        _check(load().cme_checkpoint_size(self.handle, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(load().cme_checkpoint_save(self.handle, buf, n))
        return buf.raw

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(load().cme_checkpoint_load(self.handle, buf, len(blob)))

    def transform(self, sign: int) -> np.ndarray:
        out = np.empty(2 * self.total, dtype=np.float64)
        _check(load().cme_transform(self.handle, int(sign), _dptr(out), HOST))
        return out.view(np.complex128)

    def grad(self, h: float, nsteps: int, target, eps: float = 1e-20, segment: int = 0) -> dict:
        """cme_grad: loss and gradients of the log-power-spectrum misfit after nsteps steps of
        the batch's integrator (RK4IP or Strang) from the current field (the batch ends at the
        final field)."""
        T = np.ascontiguousarray(target, dtype=np.float64).reshape(-1)
        assert T.size == self.total
        C, M = self.count, self.total
        out = {"loss": np.zeros(C), "d_sigma": np.zeros(C), "d_A_in": np.zeros(2 * C),
               "d_D2": np.zeros(C), "d_D3": np.zeros(C), "d_omega": np.zeros(M),
               "d_kappa": np.zeros(M), "d_D0": np.zeros(2 * M)}
        g = Grads(**{k: _dptr(v) for k, v in out.items()})
        _check(load().cme_grad(self.handle, float(h), int(nsteps), _dptr(T), float(eps),
                               int(segment), ctypes.byref(g)))
        # which schedule the library chose: "stored" trajectory or "checkpoint" and recompute
        self.last_grad_schedule = "stored" if g.stored else "checkpoint"
        out["d_A_in"] = out["d_A_in"].view(np.complex128)
        out["d_D0"] = out["d_D0"].view(np.complex128)
        return out

    def set_grad_memory(self, max_bytes: int):
        """cme_set_grad_memory: budget of the stored-trajectory gradient (-1 automatic, 0 never:
        checkpoint and recompute)."""
        _check(load().cme_set_grad_memory(self.handle, int(max_bytes)))

    def eval_rhs(self) -> np.ndarray:
        out = np.empty(2 * self.total, dtype=np.float64)
        _check(load().cme_eval_rhs(self.handle, _dptr(out), HOST))
        return out.view(np.complex128)


def rk4ip_noalloc(N: int, count: int, h: float, nsteps: int, d_kappa: int, d_omega: int,
                  d_inst: int, d_field: int, stream: int = 0):
    """cme_rk4ip_noalloc on device pointers supplied by the caller (no device allocation by
    the library; see include/cme.h for the 16 MiB scratch limit and the sharing rules)."""
    _check(load().cme_rk4ip_noalloc(int(N), int(count), float(h), int(nsteps), d_kappa,
                                    d_omega, d_inst, d_field, stream or None))


def fma_peak(precision=FP32) -> float:
    v = ctypes.c_double()
    _check(load().cme_fma_peak(int(precision), ctypes.byref(v)))
    return v.value


def l2_peak(nbytes: int = 16 << 20) -> float:
    """cme_l2_peak: copy bandwidth (read + write bytes/s) of an L2-resident buffer."""
    v = ctypes.c_double()
    _check(load().cme_l2_peak(int(nbytes), ctypes.byref(v)))
    return v.value


def kernel_launches() -> int:
    return int(load().cme_kernel_launches())


# ---- autograd ----------------------------------------------------------------------------------
def _autograd_function():
    import torch

    class LogSpectrumLoss(torch.autograd.Function):
        """Sum over a batch of the log-power-spectrum misfit after nsteps RK4IP steps, as a
        differentiable function of (sigma, Re A_in, Im A_in, D2, D3, Re D0, Im D0) per
        instance.  The forward pass and the discrete adjoint both run in the CUDA library
        (cme_grad); this class only marshals tensors (float64, CPU) to and from it."""

        @staticmethod
        def forward(ctx, sigma, a_re, a_im, D2, D3, d0_re, d0_im, spec):
            B, N = d0_re.shape
            mu = np.arange(N) - N // 2
            insts = []
            for b in range(B):
                om = float(D2[b]) * mu * mu / 2.0 + float(D3[b]) * mu ** 3 / 6.0
                D0 = d0_re[b].detach().numpy() + 1j * d0_im[b].detach().numpy()
                insts.append(Instance(N, np.full(N, spec["kappa"]), om, spec["g0"],
                                      spec["kappa_ext"], complex(float(a_re[b]), float(a_im[b])),
                                      float(sigma[b]), D0))
            batch = Batch(insts, precision=spec.get("precision", FP64))
            g = batch.grad(spec["h"], spec["nsteps"], spec["target"], spec.get("eps", 1e-20),
                           spec.get("segment", 0))
            batch.close()
            t = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)
            dD0 = g["d_D0"].reshape(B, N)
            ctx.save_for_backward(t(g["d_sigma"]), t(g["d_A_in"].real), t(g["d_A_in"].imag),
                                  t(g["d_D2"]), t(g["d_D3"]), t(dD0.real), t(dD0.imag))
            return t(g["loss"]).sum()

        @staticmethod
        def backward(ctx, go):
            return tuple(go * x for x in ctx.saved_tensors) + (None,)

    return LogSpectrumLoss


_LSL = None


def log_spectrum_loss(sigma, a_re, a_im, D2, D3, d0_re, d0_im, *, kappa, kappa_ext, g0, h,
                      nsteps, target, precision=FP64, eps=1e-20, segment=0):
    """Differentiable (torch.autograd) batch loss; see LogSpectrumLoss."""
    global _LSL
    if _LSL is None:
        _LSL = _autograd_function()
    spec = dict(kappa=kappa, kappa_ext=kappa_ext, g0=g0, h=h, nsteps=nsteps, target=target,
                precision=precision, eps=eps, segment=segment)
    return _LSL.apply(sigma, a_re, a_im, D2, D3, d0_re, d0_im, spec)
