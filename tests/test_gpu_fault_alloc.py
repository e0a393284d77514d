"""Failure detection by host-side fault injection: with LBM_FAULT_ALLOC=k
set when a context is created, that context's k-th device allocation
reports out of memory without allocating (no GPU fault is involved).  For
every k up to the number of allocations a full use of the library makes,
exactly one call must return LBM_ERR_NOMEM with a message, the context must
stay consistent afterwards (a geometry that failed to load leaves no
geometry behind, so steps are refused instead of running on freed tables),
and repeating the failed call once the injection is spent must succeed."""
import os

import numpy as np
import pytest

from paper_2203_01316_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LBM_ERR_NOMEM, LBM_ERR_STATE = 2, 5


def _calls(s, w, torch):
    """The library's allocating calls, in an order a user makes them."""
    N = s.N
    F, H = s.flow_record_size()
    rec = torch.empty(F + H, dtype=torch.float32, device="cuda")
    mu = torch.zeros(27 * N, dtype=torch.float32, device="cuda")
    out = torch.empty_like(mu)
    return [
        ("geometry", lambda: s.set_geometry(w["flags"], w["links"], n_walls=w["nwalls"])),
        ("source", lambda: s.set_source(w["theta"].astype(np.float32))),
        ("init", lambda: s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])),
        ("step", lambda: s.step(2)),
        ("macros", lambda: s.macros()),
        ("populations", lambda: s.populations()),
        ("stream_map", lambda: s.stream_map()),
        ("record_pre", lambda: s.step_record_pre(1, rec[:F], rec[F:])),
        ("flow_adjoint", lambda: s.adjoint_flow_step(rec[:F], rec[F:], mu, mu, out, out.clone())),
    ]


def _run(k, w):
    import torch
    from paper_2203_01316_gb300 import LBMError, Solver
    nx, ny, nz = w["dims"]
    failures = []
    os.environ["LBM_FAULT_ALLOC"] = str(k)
    try:
        try:
            s = Solver(nx, ny, nz, nu=0.03, k=2e-3, storage="f32", periodic_x=True)
        except LBMError as e:
            assert e.status == LBM_ERR_NOMEM and "out of device memory" in str(e)
            return ["create"]
    finally:
        del os.environ["LBM_FAULT_ALLOC"]
    for name, call in _calls(s, w, torch):
        try:
            call()
        except LBMError as e:
            assert e.status == LBM_ERR_NOMEM and "out of device memory" in str(e), (name, e)
            failures.append(name)
            if name == "geometry":
                with pytest.raises(LBMError) as st:
                    s.step(1)
                assert st.value.status == LBM_ERR_STATE
            call()  # the injection is spent: the same call now succeeds
            if name == "geometry":
                s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    s.sync()
    m, e = s.balances()
    assert np.isfinite(m) and np.isfinite(e)
    s.close()
    return failures


def test_every_device_allocation_failure_is_reported_and_recoverable():
    w = I.plate_channel(nx=12, ny=10, nz=6, q_bottom=0.3, q_top=0.7, theta_max=1e-3, seed=5)
    seen = []
    for k in range(1, 64):
        f = _run(k, w)
        assert len(f) <= 1, (k, f)
        if not f:
            break
        seen.append(f[0])
    else:
        pytest.fail("more than 63 allocations: extend the sweep")
    # every allocating call was reached by some k
    for name in ("create", "geometry", "source", "init", "populations", "stream_map", "flow_adjoint"):
        assert name in seen, (name, seen)
