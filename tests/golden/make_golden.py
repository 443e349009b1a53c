"""Writes the stored oracle values used by the full-size parity tests.

Calls only the CPU oracle (oracle/) on inputs from the seeded generator; no
value here comes from the CUDA path.  Each file records a hash of its inputs
so a test can confirm that it regenerates the same walkers and parameters.

    python tests/golden/make_golden.py c8h10 64
    python tests/golden/make_golden.py c26h24 16 4     # 4 processes, one walker each at a time
    python tests/golden/make_golden.py c26h24 16 grad
    python tests/golden/make_golden.py c8h10 cond local   # add cond_dominant to an existing file
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import fire_oracle as O  # noqa: E402
from paper_2504_06087_gb300 import synth  # noqa: E402


def input_hash(r, params) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(r).tobytes())
    for k in sorted(params):
        h.update(k.encode())
        h.update(np.ascontiguousarray(params[k]).tobytes())
    return h.hexdigest()


def input_summary(r, params):
    """Moments of the inputs: platform libm differences may move the last bit
    of a generated value, so tests compare these within 1e-12 instead of the
    bitwise hash."""
    out = {"r_sum": float(np.sum(r)), "r_sq": float(np.sum(r * r)), "r_first": np.ravel(r)[:6].tolist()}
    for k in sorted(params):
        out["p_" + k] = [float(np.sum(params[k])), float(np.sum(params[k] ** 2))]
    return out


def _one_walker(args):
    """Oracle local energy of walker b alone (a process of its own: the dense
    second-derivative graph of one C26H24 walker holds several GB)."""
    key, nw, b, threads = args
    torch.set_num_threads(threads)
    w = synth.workload(key)
    r, p = synth.make_inputs(w, nw)
    return O.local_energy(w.system, w.arch, p, r[b:b + 1], return_parts=True)


def main(key: str, nw: int, procs: int = 1):
    w = synth.workload(key)
    r, p = synth.make_inputs(w, nw)
    t0 = time.time()
    if procs <= 1:
        e, la, sg, kin, v, g, lap = O.local_energy(w.system, w.arch, p, r, return_parts=True)
    else:
        import concurrent.futures as cf
        import multiprocessing as mp
        threads = max(1, (os.cpu_count() or 1) // procs)
        with cf.ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_one_walker, [(key, nw, b, threads) for b in range(nw)]))
        e, la, sg, kin, v, g, lap = (np.concatenate([q[k] for q in parts]) for k in range(7))
    out = {
        "workload": key,
        "n_walkers": nw,
        "input_sha256": input_hash(r, p),
        "input_summary": input_summary(r, p),
        "source": "oracle/fire_oracle.py local_energy (FP64, dense, autograd Laplacian)",
        "seconds": time.time() - t0,
        "e_loc": e.tolist(), "logabs": la.tolist(), "sign": sg.tolist(),
        "e_kin": kin.tolist(), "e_pot": v.tolist(), "lap": lap.tolist(),
        "grad_norm2": (g ** 2).sum(axis=(1, 2)).tolist(),
        "cond_dominant": dominant_conditioning(w, r, p).tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{key}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["seconds"])




def main_grad(key: str, nw: int, nidx: int = 64):
    """Oracle d log|Psi| / d theta at nidx seeded flat indices, per walker."""
    w = synth.workload(key)
    r, p = synth.make_inputs(w, nw)
    spec = synth.param_spec(w.system, w.arch)
    sizes = [int(np.prod(s)) for _, s in spec]
    offs = np.cumsum([0] + sizes[:-1])
    idx = np.sort(np.random.default_rng(4).choice(int(sum(sizes)), size=nidx, replace=False))
    t0 = time.time()
    g = O.grad_logpsi(w.system, w.arch, p, r)
    flat = np.concatenate([g[name].reshape(nw, -1) for name, _ in spec], axis=1)
    out = {"workload": key, "n_walkers": nw, "input_sha256": input_hash(r, p),
           "input_summary": input_summary(r, p),
           "source": "oracle/fire_oracle.py grad_logpsi (FP64, autograd)", "seconds": time.time() - t0,
           "flat_index": idx.tolist(), "grad": flat[:, idx].tolist(),
           "cond_dominant": dominant_conditioning(w, r, p).tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{key}_grad_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["seconds"])


def dominant_conditioning(w, r, p) -> np.ndarray:
    """2-norm condition number of each walker's orbital matrix with the
    largest |det| (the one that dominates log|Psi| and its gradient)."""
    pt = O.params_to_torch(p)
    with torch.no_grad():
        rt = torch.as_tensor(r, dtype=torch.float64)
        _, _, h = O.embeddings(w.system, w.arch, pt, rt)
        phi = O.orbitals(w.system, w.arch, pt, rt, h).numpy()       # [W, D, n, n]
    dom = np.linalg.slogdet(phi)[1].argmax(axis=1)
    return np.array([np.linalg.cond(phi[b, dom[b]]) for b in range(phi.shape[0])])


def add_conditioning(key: str, kind: str = "grad"):
    """Adds cond_dominant to an existing {key}_grad_oracle.json or (kind
    "local") {key}_oracle.json (same inputs)."""
    name = f"{key}_grad_oracle.json" if kind == "grad" else f"{key}_oracle.json"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    out = json.load(open(path))
    w = synth.workload(key)
    r, p = synth.make_inputs(w, out["n_walkers"])
    assert input_hash(r, p) == out["input_sha256"]
    out["cond_dominant"] = dominant_conditioning(w, r, p).tolist()
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["cond_dominant"])


if __name__ == "__main__":
    if len(sys.argv) > 2 and sys.argv[2] == "cond":
        add_conditioning(sys.argv[1], sys.argv[3] if len(sys.argv) > 3 else "grad")
        sys.exit(0)
    if len(sys.argv) > 3 and sys.argv[3] == "grad":
        main_grad(sys.argv[1], int(sys.argv[2]))
    else:
        main(sys.argv[1], int(sys.argv[2]), int(sys.argv[3]) if len(sys.argv) > 3 else 1)
