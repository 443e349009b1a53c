"""Python binding of libfire (include/fire.h): argument marshalling only.

Every step of the computation runs in the CUDA kernels of libfire.so; this
module only converts arguments (ctypes structs, device pointers of torch
tensors, the current CUDA stream) and allocates the caller-owned workspace
with torch.  If libfire.so is missing the import of ``lib()`` raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfire.so")

PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
OP_NEIGHBORS, OP_LOGPSI, OP_LOCAL_ENERGY, OP_GRAD_LOGPSI, OP_MCMC = 0, 1, 2, 3, 4

STATUS = {0: "FIRE_OK", 1: "FIRE_ERR_INVALID_ARG", 2: "FIRE_ERR_CAPACITY", 3: "FIRE_ERR_NONFINITE",
          4: "FIRE_ERR_SINGULAR_REFRESH", 5: "FIRE_ERR_TIMEOUT", 6: "FIRE_ERR_CUDA",
          7: "FIRE_ERR_UNSUPPORTED", 8: "FIRE_ERR_WORKSPACE"}


class FireError(RuntimeError):
    def __init__(self, code: int, where: str, info=None):
        self.code = code
        self.info = info
        msg = f"{where}: {STATUS.get(code, code)} ({lib().fire_status_string(code).decode()})"
        if code == 6:
            msg += " last error: " + lib().fire_last_error().decode()
        super().__init__(msg)


class System(ctypes.Structure):
    _fields_ = [("n_el", ctypes.c_int32), ("n_up", ctypes.c_int32), ("n_nuc", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("nuc_pos", ctypes.c_void_p), ("nuc_charge", ctypes.c_void_p),
                ("cutoff", ctypes.c_double), ("cutoff_nuc", ctypes.c_double)]


class Arch(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("n_layers", ctypes.c_int32), ("n_det", ctypes.c_int32),
                ("n_env", ctypes.c_int32), ("n_gauss", ctypes.c_int32), ("edge_hidden", ctypes.c_int32),
                ("jastrow_width", ctypes.c_int32), ("n_reg", ctypes.c_int32), ("d_reg", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class Params(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_void_p), ("n_params", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class ParamEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("offset", ctypes.c_int64), ("ndim", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("shape", ctypes.c_int64 * 5)]


class WsEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("offset", ctypes.c_int64), ("bytes", ctypes.c_int64)]


class ProfEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("ms_total", ctypes.c_double)]


class Ecp(ctypes.Structure):
    _fields_ = [("n_quad", ctypes.c_int32), ("n_channels", ctypes.c_int32), ("n_terms", ctypes.c_int32 * 3),
                ("pad_", ctypes.c_int32), ("r_cut", ctypes.c_double), ("coef", (ctypes.c_double * 4) * 3),
                ("power", (ctypes.c_double * 4) * 3), ("alpha", (ctypes.c_double * 4) * 3)]


def ecp_table(entries):
    """fire_ecp_t array from per-nucleus entries: None (no pseudopotential) or
    {"n_quad": 4|6|12, "r_cut": x, "terms": [[(coef, power, alpha), ...] per channel l]}."""
    arr = (Ecp * len(entries))()
    for m, e in enumerate(entries):
        if e is None:
            continue
        arr[m].n_quad = int(e["n_quad"])
        arr[m].r_cut = float(e["r_cut"])
        arr[m].n_channels = len(e["terms"])
        for l, terms in enumerate(e["terms"]):
            arr[m].n_terms[l] = len(terms)
            for j, (c, pw, a) in enumerate(terms):
                arr[m].coef[l][j] = float(c)
                arr[m].power[l][j] = float(pw)
                arr[m].alpha[l][j] = float(a)
    return arr


class Info(ctypes.Structure):
    _fields_ = [("k_required", ctypes.c_int32), ("n_nodes", ctypes.c_int32), ("n_nonfinite", ctypes.c_int32),
                ("n_chunks", ctypes.c_int32), ("rows_total", ctypes.c_int64), ("mean_neighbors", ctypes.c_double),
                ("n_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
P = ctypes.POINTER
VP = ctypes.c_void_p

# name -> (restype, argtypes); mirrors include/fire.h
SIGNATURES = {
    "fire_version": (ctypes.c_char_p, []),
    "fire_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fire_last_error": (ctypes.c_char_p, []),
    "fire_param_count": (ctypes.c_int64, [P(System), P(Arch)]),
    "fire_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "fire_profile_reset": (ctypes.c_int, []),
    "fire_profile_report": (ctypes.c_int, [P(ProfEntry), P(ctypes.c_int32)]),
    "fire_param_layout": (ctypes.c_int, [P(System), P(Arch), P(ParamEntry), P(ctypes.c_int32)]),
    "fire_workspace_size": (ctypes.c_size_t, [P(System), P(Arch), ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32]),
    "fire_workspace_layout": (ctypes.c_int, [P(System), P(Arch), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, P(WsEntry), P(ctypes.c_int32), P(ctypes.c_int64)]),
    "fire_selftest_tc_gemm": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, VP, VP,
                                             VP, VP, VP]),
    "fire_selftest_fma_rate": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, VP, VP]),
    "fire_spring_workspace_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    "fire_spring_step": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, VP, ctypes.c_int64, VP, VP, ctypes.c_double,
                                        ctypes.c_double, VP, VP, VP, VP, ctypes.c_size_t, VP]),
    "fire_ecp_nonlocal": (ctypes.c_int, [P(System), P(Arch), P(Params), ctypes.c_int64, VP, ctypes.c_int32,
                                         ctypes.c_int32, P(Ecp), ctypes.c_uint64, VP, P(Info), VP, ctypes.c_size_t, VP]),
    "fire_spin_ratios": (ctypes.c_int, [P(System), P(Arch), P(Params), ctypes.c_int64, VP, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, VP, VP, P(Info), VP, ctypes.c_size_t, VP]),
    "fire_neighbors": (ctypes.c_int, [P(System), ctypes.c_int64, VP, ctypes.c_int32, VP, VP,
                                      P(ctypes.c_int32), VP, ctypes.c_size_t, VP]),
    "fire_logpsi": (ctypes.c_int, [P(System), P(Arch), P(Params), ctypes.c_int64, VP, ctypes.c_int32,
                                   ctypes.c_int32, VP, VP, P(Info), VP, ctypes.c_size_t, VP]),
    "fire_local_energy": (ctypes.c_int, [P(System), P(Arch), P(Params), ctypes.c_int64, VP, ctypes.c_int32,
                                         ctypes.c_int32, VP, VP, VP, VP, VP, P(Info), VP, ctypes.c_size_t, VP]),
    "fire_grad_logpsi": (ctypes.c_int, [P(System), P(Arch), P(Params), ctypes.c_int64, VP, ctypes.c_int32,
                                        ctypes.c_int32, VP, VP, VP, P(Info), VP, ctypes.c_size_t, VP]),
    "fire_local_energy_static": (ctypes.c_int, [P(System), P(Arch), P(Params), ctypes.c_int64, VP,
                                                ctypes.c_int32, ctypes.c_int32, VP, VP, VP, VP, VP, P(Info), VP]),
    "fire_mcmc_step": (ctypes.c_int, [P(System), P(Arch), P(Params), ctypes.c_int64, VP, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_uint64, P(ctypes.c_uint64), VP, VP, VP, P(ctypes.c_int64),
                                      P(ctypes.c_double), P(Info), VP, ctypes.c_size_t, VP]),
}

# Bytes of the library-owned workspace of fire_local_energy_static (include/fire.h).
STATIC_WORKSPACE_BYTES = 32 * 1024 * 1024


def lib():
    """Loads libfire.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2504_06087_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def profile(on: bool = True):
    L = lib()
    L.fire_profile_reset()
    L.fire_profile_enable(1 if on else 0)


def profile_report():
    """{stage: (launches, total ms)} accumulated on this host thread."""
    L = lib()
    n = ctypes.c_int32(0)
    L.fire_profile_report(None, ctypes.byref(n))
    ents = (ProfEntry * max(n.value, 1))()
    L.fire_profile_report(ents, ctypes.byref(n))
    return {e.name.decode(): (int(e.launches), float(e.ms_total)) for e in ents[:n.value]}


def split_bf16(x: torch.Tensor, nc: int) -> torch.Tensor:
    """[nc, *x.shape] bf16 components with x ~ sum of components."""
    out, r = [], x.float()
    for _ in range(nc):
        h = r.to(torch.bfloat16)
        out.append(h)
        r = r - h.float()
    return torch.stack(out)


def tc_gemm_selftest(A: torch.Tensor, Bt: torch.Tensor, nc: int = 1) -> torch.Tensor:
    """C = A @ Bt^T on the tensor cores.  A [nc, M, K] / Bt [nc, N, K] bf16
    components (or [M, K] / [N, K] for nc = 1)."""
    if A.dim() == 2:
        A, Bt = A[None], Bt[None]
    _, M, K = A.shape
    N = Bt.shape[1]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = lib().fire_selftest_tc_gemm(M, N, K, nc, _ptr(A.contiguous()), _ptr(Bt.contiguous()), _ptr(C), _ptr(err),
                                     ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream))
    torch.cuda.synchronize(A.device)
    if rc:
        raise FireError(rc, "fire_selftest_tc_gemm")
    if int(err.item()):
        raise RuntimeError(f"tensor-core product: bounded wait gave up (code {int(err.item())})")
    return C


def fma_probe(dtype: torch.dtype, iters: int, blocks: int, device="cuda") -> int:
    """Launches the SIMT multiply-add probe on the current stream (not
    synchronised; the caller times it).  Returns the FLOPs of the launch."""
    out = torch.empty(blocks * 256, dtype=dtype, device=device)
    code = 0 if dtype == torch.float64 else 1
    rc = lib().fire_selftest_fma_rate(code, iters, blocks, _ptr(out),
                                      ctypes.c_void_p(torch.cuda.current_stream(out.device).cuda_stream))
    if rc:
        raise FireError(rc, "fire_selftest_fma_rate")
    rounds = (iters + 3) // 4
    return 2 * 8 * 4 * rounds * blocks * 256


def spring_step(O: torch.Tensor, e_loc: torch.Tensor, delta_prev: Optional[torch.Tensor] = None,
                eta: float = 0.99, lam: float = 1e-3, want_gram: bool = False, want_x: bool = False,
                check: bool = True):
    """fire_spring_step on device tensors: O [N, P] float32 (row stride may
    exceed P), e_loc [N] float64, delta_prev [P] float32 or None.  Returns
    {"delta" [P] float32, "gram" [N, N] float64 or None, "x" [N] float64 or
    None, "status"}."""
    assert O.dtype == torch.float32 and O.dim() == 2 and O.stride(1) == 1
    N, Pn = O.shape
    dev = O.device
    e = e_loc.to(device=dev, dtype=torch.float64).contiguous()
    dp = None if delta_prev is None else delta_prev.to(device=dev, dtype=torch.float32).contiguous()
    delta = torch.empty(Pn, dtype=torch.float32, device=dev)
    gram = torch.empty((N, N), dtype=torch.float64, device=dev) if want_gram else None
    x = torch.empty(N, dtype=torch.float64, device=dev) if want_x else None
    nbytes = int(lib().fire_spring_workspace_size(N, Pn))
    if nbytes == 0:
        raise FireError(1, "fire_spring_workspace_size")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    rc = lib().fire_spring_step(N, Pn, _ptr(O), O.stride(0), _ptr(e), _ptr(dp), float(eta), float(lam), _ptr(delta),
                                _ptr(gram), _ptr(x), _ptr(ws), ws.numel(),
                                ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    if check and rc != 0:
        raise FireError(rc, "fire_spring_step")
    return {"delta": delta, "gram": gram, "x": x, "status": rc}


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_arch(a) -> Arch:
    return Arch(a.width, a.n_layers, a.n_det, a.n_env, a.n_gauss, a.edge_hidden, a.jastrow_width,
                a.n_reg, a.d_reg, a.flags)


def param_layout(system_c: System, arch_c: Arch):
    L = lib()
    n = ctypes.c_int32(0)
    rc = L.fire_param_layout(ctypes.byref(system_c), ctypes.byref(arch_c), None, ctypes.byref(n))
    if rc:
        raise FireError(rc, "fire_param_layout")
    ents = (ParamEntry * n.value)()
    rc = L.fire_param_layout(ctypes.byref(system_c), ctypes.byref(arch_c), ents, ctypes.byref(n))
    if rc:
        raise FireError(rc, "fire_param_layout")
    return [(e.name.decode(), int(e.offset), tuple(int(e.shape[k]) for k in range(e.ndim))) for e in ents]


class Fire:
    """A molecule, a network and its parameters resident on one CUDA device."""

    def __init__(self, system, arch, params: Dict[str, np.ndarray], precision: str = "fp32",
                 k_cap: int = 64, device: str = "cuda:0"):
        self.system, self.arch, self.precision = system, arch, precision
        self.prec = PREC[precision]
        self.k_cap = int(k_cap)
        self.device = torch.device(device)
        self.nuc_pos = torch.as_tensor(np.ascontiguousarray(system.nuc_pos), dtype=torch.float64,
                                       device=self.device)
        self.nuc_charge = torch.as_tensor(np.ascontiguousarray(system.nuc_charge), dtype=torch.float64,
                                          device=self.device)
        self.sys_c = System(system.n_el, system.n_up, system.n_nuc, 0, self.nuc_pos.data_ptr(),
                            self.nuc_charge.data_ptr(), float(system.cutoff), float(system.cutoff_nuc))
        self.arch_c = make_arch(arch)
        self.layout = param_layout(self.sys_c, self.arch_c)
        self.n_params = int(lib().fire_param_count(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c)))
        self.set_params(params)
        self._ws = {}

    def set_params(self, params: Dict[str, np.ndarray]):
        dt = np.float64 if self.prec == 0 else np.float32
        flat = np.zeros(self.n_params, dtype=dt)
        for name, off, shape in self.layout:
            a = np.asarray(params[name])
            if tuple(a.shape) != tuple(shape):
                raise ValueError(f"parameter {name}: shape {a.shape} != {shape}")
            flat[off:off + a.size] = a.reshape(-1)
        self.theta = torch.as_tensor(flat, device=self.device)
        self.params_c = Params(self.theta.data_ptr(), self.n_params, 0 if self.prec == 0 else 1, 0)

    def set_theta(self, theta: torch.Tensor):
        """Use a flat device parameter tensor (layout of fire_param_layout) as theta."""
        dt = torch.float64 if self.prec == 0 else torch.float32
        t = theta.detach().to(device=self.device, dtype=dt).contiguous()
        assert t.numel() == self.n_params
        self.theta = t
        self.params_c = Params(self.theta.data_ptr(), self.n_params, 0 if self.prec == 0 else 1, 0)

    def workspace(self, W: int, op: int) -> torch.Tensor:
        key = (W, op)
        if key not in self._ws:
            nbytes = lib().fire_workspace_size(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c), W,
                                               self.prec, self.k_cap, op)
            if nbytes == 0:
                raise FireError(1, "fire_workspace_size")
            self._ws = {key: torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)}
        return self._ws[key]

    def workspace_layout(self, W: int, op: int):
        """name -> (byte offset, bytes) of the intermediates of the first walker chunk."""
        L = lib()
        n, wc = ctypes.c_int32(0), ctypes.c_int64(0)
        args = (ctypes.byref(self.sys_c), ctypes.byref(self.arch_c), W, self.prec, self.k_cap, op)
        rc = L.fire_workspace_layout(*args, None, ctypes.byref(n), ctypes.byref(wc))
        if rc:
            raise FireError(rc, "fire_workspace_layout")
        ents = (WsEntry * n.value)()
        L.fire_workspace_layout(*args, ents, ctypes.byref(n), ctypes.byref(wc))
        return {e.name.decode(): (int(e.offset), int(e.bytes)) for e in ents}, int(wc.value)

    def ws_view(self, W: int, op: int, name: str, dtype, shape=None):
        """A typed view of one intermediate buffer of the last call (no copy)."""
        lay, _ = self.workspace_layout(W, op)
        off, nb = lay[name]
        ws = self.workspace(W, op)
        t = ws[off:off + nb].view(dtype)
        return t if shape is None else t[:int(np.prod(shape))].view(*shape)

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _r(self, r):
        if not isinstance(r, torch.Tensor):
            r = torch.as_tensor(np.ascontiguousarray(r), dtype=torch.float64)
        r = r.to(device=self.device, dtype=torch.float64).contiguous()
        assert r.dim() == 3 and r.shape[1] == self.system.n_el and r.shape[2] == 3
        return r

    def local_energy(self, r, check: bool = True):
        r = self._r(r)
        W = r.shape[0]
        out = {k: torch.empty(W, dtype=torch.float64, device=self.device)
               for k in ("e_loc", "logabs", "sign", "e_kin", "e_pot")}
        ws = self.workspace(W, OP_LOCAL_ENERGY)
        info = Info()
        rc = lib().fire_local_energy(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c),
                                     ctypes.byref(self.params_c), W, _ptr(r), self.k_cap, self.prec,
                                     _ptr(out["e_loc"]), _ptr(out["logabs"]), _ptr(out["sign"]),
                                     _ptr(out["e_kin"]), _ptr(out["e_pot"]), ctypes.byref(info),
                                     _ptr(ws), ws.numel(), self._stream())
        out["info"] = info.as_dict()
        out["status"] = rc
        if check and rc not in (0,):
            raise FireError(rc, "fire_local_energy", out["info"])
        return out

    def local_energy_static(self, r, check: bool = True):
        """fire_local_energy_static: the library's own static workspace, no
        device allocation inside the call (the outputs here are torch tensors
        allocated by this wrapper, as a caller would provide them)."""
        r = self._r(r)
        W = r.shape[0]
        out = {k: torch.empty(W, dtype=torch.float64, device=self.device)
               for k in ("e_loc", "logabs", "sign", "e_kin", "e_pot")}
        info = Info()
        rc = lib().fire_local_energy_static(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c),
                                            ctypes.byref(self.params_c), W, _ptr(r), self.k_cap, self.prec,
                                            _ptr(out["e_loc"]), _ptr(out["logabs"]), _ptr(out["sign"]),
                                            _ptr(out["e_kin"]), _ptr(out["e_pot"]), ctypes.byref(info),
                                            self._stream())
        out["info"] = info.as_dict()
        out["status"] = rc
        if check and rc != 0:
            raise FireError(rc, "fire_local_energy_static", out["info"])
        return out

    def logpsi(self, r, check: bool = True):
        r = self._r(r)
        W = r.shape[0]
        out = {k: torch.empty(W, dtype=torch.float64, device=self.device) for k in ("logabs", "sign")}
        ws = self.workspace(W, OP_LOGPSI)
        info = Info()
        rc = lib().fire_logpsi(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c), ctypes.byref(self.params_c),
                               W, _ptr(r), self.k_cap, self.prec, _ptr(out["logabs"]), _ptr(out["sign"]),
                               ctypes.byref(info), _ptr(ws), ws.numel(), self._stream())
        out["info"] = info.as_dict()
        out["status"] = rc
        if check and rc != 0:
            raise FireError(rc, "fire_logpsi", out["info"])
        return out

    def grad_logpsi(self, r, check: bool = True):
        """Per-walker d log|Psi| / d theta: {"grad": [W, P], "logabs", "sign"}."""
        r = self._r(r)
        W = r.shape[0]
        dt = torch.float64 if self.prec == 0 else torch.float32
        out = {"grad": torch.empty((W, self.n_params), dtype=dt, device=self.device),
               "logabs": torch.empty(W, dtype=torch.float64, device=self.device),
               "sign": torch.empty(W, dtype=torch.float64, device=self.device)}
        ws = self.workspace(W, OP_GRAD_LOGPSI)
        info = Info()
        rc = lib().fire_grad_logpsi(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c),
                                    ctypes.byref(self.params_c), W, _ptr(r), self.k_cap, self.prec,
                                    _ptr(out["grad"]), _ptr(out["logabs"]), _ptr(out["sign"]), ctypes.byref(info),
                                    _ptr(ws), ws.numel(), self._stream())
        out["info"] = info.as_dict()
        out["status"] = rc
        if check and rc != 0:
            raise FireError(rc, "fire_grad_logpsi", out["info"])
        return out

    def mcmc_step(self, r: torch.Tensor, sigma: float, n_sweeps: int, refresh_every: int = 32, seed: int = 0,
                  counter: int = 0, check: bool = True, n_global: int = 0, sigma_global: float = 2.0):
        """fire_mcmc_step: n_sweeps Metropolis sweeps of single-electron moves on
        the device positions r [W, n_el, 3] float64, updated in place; each
        sweep ends with n_global global jumps (mixture width sigma_global).
        Returns {"logabs", "sign", "accepted" [W], "n_accepted", "max_drift",
        "counter" (the advanced move counter), "info", "status"}."""
        assert isinstance(r, torch.Tensor) and r.dtype == torch.float64 and r.is_contiguous()
        assert r.device == torch.device(self.device) and r.dim() == 3 and r.shape[1] == self.system.n_el
        W = r.shape[0]
        out = {k: torch.empty(W, dtype=torch.float64, device=self.device) for k in ("logabs", "sign")}
        out["accepted"] = torch.empty(W, dtype=torch.int32, device=self.device)
        ws = self.workspace(W, OP_MCMC)
        info = Info()
        ctr = ctypes.c_uint64(counter)
        nacc = ctypes.c_int64(0)
        drift = ctypes.c_double(0.0)
        rc = lib().fire_mcmc_step(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c), ctypes.byref(self.params_c),
                                  W, _ptr(r), self.k_cap, self.prec, float(sigma), int(n_sweeps),
                                  int(refresh_every), int(n_global), float(sigma_global),
                                  ctypes.c_uint64(seed), ctypes.byref(ctr), _ptr(out["logabs"]),
                                  _ptr(out["sign"]), _ptr(out["accepted"]), ctypes.byref(nacc),
                                  ctypes.byref(drift), ctypes.byref(info), _ptr(ws), ws.numel(), self._stream())
        out.update({"n_accepted": int(nacc.value), "max_drift": float(drift.value), "counter": int(ctr.value),
                    "info": info.as_dict(), "status": rc})
        # per-walker largest drift of this call (a diagnostic buffer of the workspace)
        out["walker_drift"] = self.ws_view(W, OP_MCMC, "mc_wdrift", torch.float64, (W,)).clone()
        # diagnostic counters of the call: ratios from a float64 LU, refactorised determinants
        stat = self.ws_view(W, OP_MCMC, "mc_stat", torch.int64, (4,)).cpu().numpy()
        out["n_exact"], out["n_repair"] = int(stat[2]), int(stat[3])
        if check and rc != 0:
            raise FireError(rc, "fire_mcmc_step", out["info"])
        return out

    def ecp_nonlocal(self, r, entries, seed: int = 0, check: bool = True):
        """fire_ecp_nonlocal: the non-local pseudopotential energy per walker
        for the per-nucleus table `entries` (see ecp_table)."""
        r = self._r(r)
        W = r.shape[0]
        v = torch.empty(W, dtype=torch.float64, device=self.device)
        tab = ecp_table(entries)
        ws = self.workspace(W, OP_MCMC)
        info = Info()
        rc = lib().fire_ecp_nonlocal(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c), ctypes.byref(self.params_c),
                                     W, _ptr(r), self.k_cap, self.prec, tab, ctypes.c_uint64(seed), _ptr(v),
                                     ctypes.byref(info), _ptr(ws), ws.numel(), self._stream())
        out = {"v_nl": v, "info": info.as_dict(), "status": rc}
        if check and rc != 0:
            raise FireError(rc, "fire_ecp_nonlocal", out["info"])
        return out

    def spin_ratios(self, r, beta: int, check: bool = True):
        """fire_spin_ratios: Psi(pi_{alpha beta} r)/Psi(r) for every spin-up
        alpha ([W, n_up]) and R_beta = 1 - their sum ([W])."""
        r = self._r(r)
        W = r.shape[0]
        ratios = torch.empty((W, self.system.n_up), dtype=torch.float64, device=self.device)
        rb = torch.empty(W, dtype=torch.float64, device=self.device)
        ws = self.workspace(W, OP_MCMC)
        info = Info()
        rc = lib().fire_spin_ratios(ctypes.byref(self.sys_c), ctypes.byref(self.arch_c), ctypes.byref(self.params_c),
                                    W, _ptr(r), self.k_cap, self.prec, int(beta), _ptr(ratios), _ptr(rb),
                                    ctypes.byref(info), _ptr(ws), ws.numel(), self._stream())
        out = {"ratios": ratios, "r_beta": rb, "info": info.as_dict(), "status": rc}
        if check and rc != 0:
            raise FireError(rc, "fire_spin_ratios", out["info"])
        return out

    def unflatten(self, flat):
        """{name: array [..., *shape]} views of a flat parameter-sized last axis."""
        return {name: flat[..., off:off + int(np.prod(shape))].reshape(*flat.shape[:-1], *shape)
                for name, off, shape in self.layout}

    def neighbors(self, r):
        r = self._r(r)
        W, n = r.shape[0], self.system.n_el
        idx = torch.full((W, n, self.k_cap), -1, dtype=torch.int32, device=self.device)
        cnt = torch.zeros((W, n, 2), dtype=torch.int32, device=self.device)
        ws = torch.empty(256, dtype=torch.uint8, device=self.device)
        kreq = ctypes.c_int32(0)
        rc = lib().fire_neighbors(ctypes.byref(self.sys_c), W, _ptr(r), self.k_cap, _ptr(idx), _ptr(cnt),
                                  ctypes.byref(kreq), _ptr(ws), ws.numel(), self._stream())
        return {"idx": idx, "cnt": cnt, "k_required": kreq.value, "status": rc}


class LogPsi(torch.autograd.Function):
    """log|Psi(r; theta)| as a differentiable function of the flat parameter
    tensor theta.  Forward: fire_logpsi.  Backward: fire_grad_logpsi (the
    adjoint kernels, embeddings recomputed) contracted with the incoming
    gradient: d/dtheta sum_w g_w log|Psi_w| = sum_w g_w O_w.  Positions get
    no gradient."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, r: torch.Tensor, model: "Fire"):
        model.set_theta(theta)
        out = model.logpsi(r)
        ctx.model = model
        ctx.save_for_backward(theta, r)
        return out["logabs"]

    @staticmethod
    def backward(ctx, g):
        theta, r = ctx.saved_tensors
        ctx.model.set_theta(theta)
        rows = ctx.model.grad_logpsi(r)["grad"]
        return (g.to(rows.dtype) @ rows).to(theta.dtype), None, None


def logpsi(theta: torch.Tensor, r: torch.Tensor, model: "Fire") -> torch.Tensor:
    return LogPsi.apply(theta, r, model)
