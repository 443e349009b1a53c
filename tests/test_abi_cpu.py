"""Host-side checks of libfire: no kernel is launched here (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2504_06087_gb300 import fire, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_or_skip():
    if not os.path.exists(fire.LIB_PATH):
        from paper_2504_06087_gb300 import build
        build.build()
    return fire.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fire_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = _lib_or_skip()
    names = declared_functions()
    assert "fire_local_energy" in names and "fire_logpsi" in names and "fire_neighbors" in names
    for nm in names:
        assert hasattr(L, nm), nm
    assert L.fire_version().startswith(b"libfire")


def _c_structs(key):
    w = synth.workload(key)
    s = w.system
    sys_c = fire.System(s.n_el, s.n_up, s.n_nuc, 0, None, None, s.cutoff, s.cutoff_nuc)
    return w, sys_c, fire.make_arch(w.arch)


@pytest.mark.parametrize("key", ["water", "c8h10", "c26h24"])
def test_param_layout_matches_generator(key):
    _lib_or_skip()
    w, sys_c, arch_c = _c_structs(key)
    lay = fire.param_layout(sys_c, arch_c)
    spec = synth.param_spec(w.system, w.arch)
    assert [(n, s) for n, _, s in lay] == [(n, tuple(s)) for n, s in spec]
    offs = [o for _, o, _ in lay]
    sizes = [int(np.prod(s)) for _, s in spec]
    assert offs == list(np.cumsum([0] + sizes[:-1]))
    total = fire.lib().fire_param_count(ctypes.byref(sys_c), ctypes.byref(arch_c))
    assert total == sum(sizes)


def test_workspace_size_and_chunking(monkeypatch):
    _lib_or_skip()
    w, sys_c, arch_c = _c_structs("c26h24")
    L = fire.lib()
    a = L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 4096, 2, 64, fire.OP_LOCAL_ENERGY)
    b = L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 4, 2, 64, fire.OP_LOCAL_ENERGY)
    c = L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 4, 2, 64, fire.OP_LOGPSI)
    assert a > b > c > 0
    assert a <= 130 * 2 ** 30         # the default budget (128 GiB) bounds a chunk
    # invalid arguments -> 0
    assert L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 0, 2, 64, 2) == 0
    assert L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 4, 7, 64, 2) == 0


def test_lu_panel_limit_is_reported_on_the_host():
    """The float64 LU keeps a panel and the U12 block of n rows in shared
    memory ((2 * 16 + 1) n doubles <= 227 KB, so n <= 880): a larger system is
    rejected by the plan (workspace size 0), a system just below runs."""
    _lib_or_skip()
    L = fire.lib()
    arch_c = fire.make_arch(synth.workload("c26h24").arch)
    for k, ok in ((124, True), (128, False)):      # C_kH_{k+2}: n_el = 7k + 2 = 870, 898
        s = synth.zigzag_polyene(k)
        assert s.n_el == 7 * k + 2
        sys_c = fire.System(s.n_el, s.n_up, s.n_nuc, 0, None, None, s.cutoff, s.cutoff_nuc)
        size = L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 2, 2, 64, fire.OP_LOGPSI)
        assert (size > 0) == ok, (s.n_el, size)


def test_host_side_argument_errors():
    _lib_or_skip()
    w, sys_c, arch_c = _c_structs("water")
    L = fire.lib()
    info = fire.Info()
    prm = fire.Params(None, 0, 0, 0)
    # NULL theta -> invalid argument, detected before any launch
    rc = L.fire_local_energy(ctypes.byref(sys_c), ctypes.byref(arch_c), ctypes.byref(prm), 4, None, 64, 0,
                             None, None, None, None, None, ctypes.byref(info), None, 0, None)
    assert rc == 1
    bad = fire.Arch(48, 2, 4, 8, 32, 16, 0, 16, 16, 7)      # width not a multiple of 32
    assert L.fire_param_count(ctypes.byref(sys_c), ctypes.byref(bad)) == -1
    odd = fire.Arch(64, 2, 4, 8, 24, 16, 0, 16, 16, 7)      # d_0 != 32 is not built
    n = ctypes.c_int32(0)
    assert L.fire_param_layout(ctypes.byref(sys_c), ctypes.byref(odd), None, ctypes.byref(n)) == 7
    assert L.fire_status_string(2).decode().startswith("neighbour")


def test_mcmc_host_side_argument_errors():
    """fire_mcmc_step rejects bad step sizes, sweep counts and missing
    pointers on the host, before any launch; its workspace holds every walker
    (no chunking) and the cached state on top of the value forward."""
    _lib_or_skip()
    w, sys_c, arch_c = _c_structs("water")
    L = fire.lib()
    prm = fire.Params(ctypes.c_void_p(16), 1, 0, 0)      # never dereferenced: rejected first
    ctr = ctypes.c_uint64(0)
    r = ctypes.c_void_p(16)
    nacc, drift, info = ctypes.c_int64(0), ctypes.c_double(0), fire.Info()

    def call(sigma=0.3, sweeps=1, refresh=32, counter=ctypes.byref(ctr), rr=r, ng=0, sg=2.0):
        return L.fire_mcmc_step(ctypes.byref(sys_c), ctypes.byref(arch_c), ctypes.byref(prm), 4, rr, 64, 0,
                                sigma, sweeps, refresh, ng, sg, 1, counter, None, None, None, ctypes.byref(nacc),
                                ctypes.byref(drift), ctypes.byref(info), None, 0, None)
    assert call(ng=-1) == 1
    assert call(ng=20, sg=0.0) == 1
    assert call(ng=20, sg=float("nan")) == 1
    assert call(sigma=0.0) == 1
    assert call(sigma=-1.0) == 1
    assert call(sigma=float("nan")) == 1
    assert call(sweeps=-1) == 1
    assert call(refresh=-2) == 1
    assert call(counter=None) == 1
    assert call(rr=None) == 1
    assert ctr.value == 0
    big = L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 4096, 1, 64, fire.OP_MCMC)
    val = L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 4096, 1, 64, fire.OP_LOGPSI)
    assert big > val > 0
    # the BF16_FP64 form samples in float32: same plan as FP32
    b16 = L.fire_workspace_size(ctypes.byref(sys_c), ctypes.byref(arch_c), 4096, 2, 64, fire.OP_MCMC)
    assert b16 == big
