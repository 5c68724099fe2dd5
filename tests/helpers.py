"""Shared test helpers: seeded scan descriptions handed to both the oracle
and the CUDA binding, and the error metrics the parity tests report."""
import json
import os

import numpy as np
import torch

import oracle as O
from paper_2103_10329_gb300 import synth

# per-ray / per-voxel relative error bound for float32 results against the
# float64 oracle: |a - o| / max(|o|, 1e-2 max|o|)
TOL_F32 = 1e-5


def scan_desc(n, nu, nv, nviews, seed, levels=1, drift=None, pitch=None, z_scale=1.0, slice_axis=2):
    th, z = synth.trajectory(nviews, seed)
    z = z * z_scale
    pitch = pitch or synth.default_pitch(nu)
    return dict(n=n, nu=nu, nv=nv, theta=th, z=z, pitch=pitch, levels=levels, drift=drift,
                slice_axis=slice_axis)


def oracle_scan(d):
    return O.Scan(n=d["n"], nu=d["nu"], nv=d["nv"], theta=d["theta"], z=d["z"], pitch=d["pitch"],
                  drift=d["drift"], slice_axis=d["slice_axis"])


def gpu_geom(d):
    from paper_2103_10329_gb300 import mgct
    return mgct.Geometry(d["n"], d["nu"], d["nv"], d["theta"], d["z"], d["pitch"], levels=d["levels"],
                         drift=d["drift"], p_slice_axis=d["slice_axis"])


def rel_err(got, ref, floor_frac=1e-2):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.maximum(np.abs(ref), floor_frac * np.abs(ref).max())
    return np.abs(got - ref) / den


def summary(e):
    return f"p50={np.percentile(e, 50):.2e} p99={np.percentile(e, 99):.2e} max={e.max():.2e}"


def check_err(e, tol, bound="max"):
    """Asserts max(e) <= tol (bound "max") or sqrt(mean(e^2)) <= tol (bound
    "rms").  With MGCT_PARITY_REPORT set to a file path, first appends the
    test's p50, p99, max and rms of e and the bound to it as one JSON line."""
    e = np.asarray(e, dtype=np.float64)
    rms = float(np.sqrt(np.mean(e ** 2))) if e.size else 0.0
    path = os.environ.get("MGCT_PARITY_REPORT")
    if path and e.size:
        rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], "n": int(e.size),
               "p50": float(np.percentile(e, 50)), "p99": float(np.percentile(e, 99)), "max": float(e.max()),
               "rms": rms, "bound": bound, "tol": float(tol)}
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")
    if bound == "max":
        assert e.max() <= tol, summary(e)
    else:
        assert rms <= tol, f"rms={rms:.2e} " + summary(e)


def to_np(t: torch.Tensor):
    return t.detach().to("cpu", torch.float64).numpy()


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")
