"""The no-allocation entry point, for callers that cannot allocate device
memory where they relax (their memory manager owns the device, or an
allocation could stall a real-time loop).  It must give what the library's
ordinary entry points give: the relaxed C-points and residual of one
FCF-relaxation, rebuilt here from mgrit_propagate and from the oracle's
relaxation, on two calls in a row that share the static scratch array, in
FP64 and MIXED.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1910_03726_gb300 import build
    build.build()
    from paper_1910_03726_gb300 import capi as c
    return c


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_fcf(c_old, taps, m):
    """The oracle's FCF-relaxation and C-point residual (Section 2.2) of a
    space-time iterate whose C-points are c_old: the relaxed C-points and
    r_j = Phi^m c'_{j-1} - c'_j after the second F-relaxation."""
    from oracle import mgrit as omg
    N = c_old.shape[0] - 1
    U = np.zeros((N * m + 1, c_old.shape[1]))
    U[::m] = c_old
    G = np.zeros_like(U)
    step = omg.stencil_step(dict(zip(taps[0], taps[1])))
    omg.f_relax(U, G, step, m)
    omg.c_relax(U, G, step, m)
    omg.f_relax(U, G, step, m)
    return U[::m], omg.c_residual(U, G, step, m)


@pytest.mark.parametrize("precision,tol", [(0, TOL), (1, 1e-6)])
def test_static_scratch_fcf_matches_library_and_oracle_two_calls(capi, precision, tol):
    """Two calls in a row on different data (the shared scratch keeps the
    first call's partial norms) against the library's ordinary entry point
    (mgrit_propagate, FP64) and the oracle's relaxation.  MIXED evaluates the
    second F-relaxation, which only acts on the correction, in FP32: its
    residual matches to FP32 rounding (1e-6 relative), its C-points exactly
    as FP64 (tolerance 1e-12)."""
    import torch
    from oracle import schemes  # only for the CFL number of the test problem

    nx, m, N, p = 320, 4, 37, 3            # nx not a power of two; ragged tail of threads
    c = schemes.cfl_number("ERK", p)
    prob = capi.problem(nx, m * N, "ERK", p, p, c)
    offs, cfs = capi.mgrit_phi_taps(prob)
    h = capi.mgrit_setup(prob, capi.mgrit_opts_default(m=m, levels=2))
    try:
        for call, seed in enumerate((5, 6)):
            rng = np.random.default_rng(seed)
            c_old_np = rng.standard_normal((N + 1, nx))
            c_old = torch.tensor(c_old_np, device="cuda")
            c_new = torch.zeros_like(c_old)
            r = torch.zeros_like(c_old)
            norm2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            capi.mgrit_fcf_residual_static(c_old, c_new, r, norm2, nx, m, N, offs, cfs, precision)
            torch.cuda.synchronize()
            # the same quantities from the library's ordinary entry point
            cn_ref = torch.zeros((N, nx), dtype=torch.float64, device="cuda")
            capi.mgrit_propagate(h, 1, m, N, c_old[:N].contiguous(), cn_ref)
            rho = (cn_ref - c_old[1:]).contiguous()
            r_ref = torch.zeros((N - 1, nx), dtype=torch.float64, device="cuda")
            capi.mgrit_propagate(h, 1, m, N - 1, rho[: N - 1].contiguous(), r_ref)
            got_c, want_c = c_new[1:].cpu().numpy(), cn_ref.cpu().numpy()
            got_r, want_r = r[2:].cpu().numpy(), r_ref.cpu().numpy()
            assert _rel(got_c, want_c) <= TOL, call
            assert _rel(got_r, want_r) <= tol, call
            want_n2 = float((r_ref * r_ref).sum())
            assert abs(float(norm2.item()) - want_n2) <= 2 * tol * want_n2, call
            assert float(c_new[0].abs().max()) == 0.0 and float(r[:2].abs().max()) == 0.0
            # and from the oracle
            oc, orr = oracle_fcf(c_old_np, (offs, cfs), m)
            assert _rel(got_c, oc[1:]) <= TOL, call
            assert _rel(got_r, orr[2:]) <= tol, call
            assert abs(float(norm2.item()) - float(np.sum(orr[2:] ** 2))) <= 2 * tol * float(np.sum(orr[2:] ** 2))
    finally:
        capi.mgrit_destroy(h)


def test_static_scratch_rejects_oversize_requests(capi):
    import torch
    nx = 64
    big = 65536 + 1
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.MgritError) as ei:
        capi.mgrit_fcf_residual_static(dummy, dummy, dummy, dummy, nx, 4, big, [0, -1], [0.15, 0.85])
    assert ei.value.status == -1
    assert "65536" in capi.mgrit_last_error()
