"""Checkpoint and resume of a solver state, and a per-solve JSONL log.

The paper restarts its runs from developed flow fields (Sec. 4) without describing the format.
Here a checkpoint is two files next to each other:

* ``<path>.f64``: the modal coefficients, raw little-endian FP64, laid out
  [element][u, v, w, p][mode] as every vector of the library;
* ``<path>.json``: a header with the mesh (cells per axis, node coordinates), the degrees of the
  p-levels, nu, c, eta, the walls flag, and the caller's time, step and 1/(gamma dt).

``load_state`` checks the header against a handle before it hands the vector back, so a state is
never resumed on another discretisation. Reloading gives the saved coefficients bit for bit.
Host I/O only: the state is copied from / to the device with one transfer each way.
"""
import json
import os

import numpy as np

FORMAT = "dgpmg-state-1"


def _header(dg, t, step, inv_gamma_dt, extra):
    p = dg.params
    hdr = {"format": FORMAT, "levels": list(dg.levels), "ne": int(dg.ne), "nb": int(dg.nb[0]),
           "nu": float(p.nu), "ac_c": float(p.ac_c), "eta": float(p.eta), "walls": int(p.walls),
           "t": float(t), "step": int(step), "inv_gamma_dt": None if inv_gamma_dt is None else float(inv_gamma_dt),
           "dtype": "<f8", "layout": "[element][u,v,w,p][mode]"}
    if dg.nprob == 1:
        hdr["cells"] = [int(p.nx), int(p.ny), int(p.nz)]
        hdr["nodes"] = [np.asarray(a, dtype=np.float64).tolist() for a in dg._nodes]
    else:
        hdr["problems"] = int(dg.nprob)
        hdr["elem_start"] = list(dg.elem_start)
    if extra:
        hdr["extra"] = extra
    return hdr


def save_state(path, w, dg, t=0.0, step=0, inv_gamma_dt=None, extra=None):
    """Write the state w (a float64 tensor or array of dg's fine-level size) to <path>.f64 and its
    header to <path>.json. Returns the header."""
    import torch
    a = w.detach().cpu().numpy() if isinstance(w, torch.Tensor) else np.asarray(w)
    a = np.ascontiguousarray(a, dtype="<f8").reshape(-1)
    if a.size != dg.n[0]:
        raise ValueError("state has %d entries, the handle's fine level %d" % (a.size, dg.n[0]))
    hdr = _header(dg, t, step, inv_gamma_dt, extra)
    hdr["entries"] = int(a.size)
    tmp = path + ".f64.tmp"
    a.tofile(tmp)
    os.replace(tmp, path + ".f64")
    with open(path + ".json.tmp", "w") as f:
        json.dump(hdr, f)
    os.replace(path + ".json.tmp", path + ".json")
    return hdr


def load_state(path, dg=None, device="cuda"):
    """Read a checkpoint: (state as a float64 tensor [ne, 4, nb] on `device`, header). With a
    handle, the header must describe the same discretisation (ValueError otherwise)."""
    import torch
    with open(path + ".json") as f:
        hdr = json.load(f)
    if hdr.get("format") != FORMAT:
        raise ValueError("not a dgpmg state file: %s" % path)
    a = np.fromfile(path + ".f64", dtype="<f8")
    if a.size != hdr["entries"]:
        raise ValueError("state file holds %d entries, its header %d" % (a.size, hdr["entries"]))
    if dg is not None:
        want = _header(dg, 0.0, 0, None, None)
        for key in ("levels", "ne", "nb", "nu", "ac_c", "eta", "walls", "cells", "nodes", "problems",
                    "elem_start"):
            if want.get(key) != hdr.get(key):
                raise ValueError("checkpoint %s differs from the handle in %r" % (path, key))
    t = torch.from_numpy(a.reshape(hdr["ne"], 4, hdr["nb"]).copy())
    return (t.to(device) if device else t), hdr


def log_solve(path, info, rc, **fields):
    """Append one JSON line describing an FGMRES solve (its, status, residuals, rho, fallback) and
    any extra fields to the file at path."""
    rec = {"rc": int(rc), "its": int(info.its), "status": int(info.status), "r0": float(info.r0),
           "relres_est": float(info.relres_est), "true_relres": float(info.true_relres), "rho": float(info.rho),
           "fallback_at": int(info.fallback_at)}
    rec.update(fields)
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")
    return rec
