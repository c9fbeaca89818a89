"""The C interface used from a plain C99 program (tests/c/gsm_c_client.c):
device and host applies and a saved-and-reloaded plan agree bit for bit, and
on the same input bits the values equal the Python binding's."""
import os
import subprocess

import numpy as np
import pytest

from test_abi import _build_c_client

pytestmark = pytest.mark.gpu


def test_c_client_matches_binding(tmp_path):
    import torch
    import paper_1501_04438_gb300 as gsm
    from paper_1501_04438_gb300 import build, workloads as wl
    libpath = build.build()
    exe = str(tmp_path / "client")
    r = _build_c_client(libpath, exe)
    assert r.returncode == 0, r.stderr
    X, Y, Z = wl.mesh((24, 20, 16), 4.0)
    rho = np.exp(-(X * X + Y * Y + Z * Z))
    rho.tofile(str(tmp_path / "rho.bin"))
    run = subprocess.run([exe, str(tmp_path / "rho.bin")], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr
    lines = run.stdout.split("\n")
    S = int(lines[0].split()[1])
    vals = {int(l.split()[1]): float(l.split()[2]) for l in lines if l.startswith("u ")}
    plan = gsm.Plan("coulomb3d", 4.0, (24, 20, 16))
    assert plan.info()["S"] == S
    u = plan.apply(torch.tensor(rho, device="cuda")).cpu().numpy().ravel()
    for i, v in vals.items():
        assert u[i] == v, (i, u[i], v)
