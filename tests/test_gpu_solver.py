"""GPU parity of the CG solve and of the monodomain time step against the oracle,
plus the solver's error reporting.

Time steps: the oracle solves each linear system exactly (sparse LU); the
GPU runs Jacobi-CG to ||r|| <= 1e-13 ||b|| so that the solution tolerance of
1e-10 (relative, 2-norm) is not consumed by the iteration.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import ionic
from oracle import mesh as Mh
from oracle import monodomain as MD

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2205_05136_gb300")
capi = gb.capi


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _small(p=2, quad="LGL", perturb=0.0, dims=(8, 4, 2)):
    s = W.slab(*dims, (20.0, 7.0, 3.0), perturb=perturb, seed=1)
    tissue = W.constant_tissue(s, 0.12, 0.03, 0.0)
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    g.set_tissue(*tissue)
    o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    return s, tissue, g, o


def test_small_slab_dof_count():
    """8 x 4 x 2 elements at p = 2: 17 x 9 x 5 = 765 nodes (the small slab workload)."""
    _, _, g, o = _small()
    assert g.ndofs == o.ndofs == 765


@pytest.mark.parametrize("quad", ["LG", "LGL"])
@pytest.mark.parametrize("precond", [capi.SEM_PC_JACOBI, capi.SEM_PC_NONE])
def test_cg_solve_matches_direct_solve(quad, precond):
    s, tissue, g, o = _small(3, quad, perturb=0.1, dims=(4, 3, 2))
    alpha = 1.5 / 0.05
    A = Mh.assemble(o, tissue, alpha, 1.0)
    b = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=3)
    import scipy.sparse.linalg as spla
    xref = spla.spsolve(A.tocsc(), b)
    x = torch.zeros(o.ndofs, dtype=torch.float64, device="cuda")
    it, res = g.cg_solve(alpha, torch.tensor(b, device="cuda"), x, rtol=1e-13, maxit=5000,
                         precond=precond)
    assert it > 0
    assert res <= 1e-13 * np.linalg.norm(b) * 1.0000001
    assert rel(x.cpu().numpy(), xref) < 1e-11


def test_cg_reports_not_converged_and_nonfinite():
    _, _, g, o = _small()
    b = torch.tensor(W.uniform_vector(o.ndofs, seed=3), device="cuda")
    x = torch.zeros_like(b)
    rc, it, res = capi.sem_cg_solve(g.ctx, 30.0, b, x, 1e-14, 0.0, 3, capi.SEM_PC_JACOBI,
                                    raise_on_error=False)
    assert rc == capi.SEM_ERR_NOT_CONVERGED and it == 3
    assert "did not converge" in capi.sem_last_error(g.ctx)
    b[5] = float("nan")
    x.zero_()
    rc, _, _ = capi.sem_cg_solve(g.ctx, 30.0, b, x, 1e-10, 0.0, 50, capi.SEM_PC_JACOBI,
                                 raise_on_error=False)
    assert rc == capi.SEM_ERR_NONFINITE


def test_argument_errors_on_gpu():
    _, _, g, o = _small()
    u_host = torch.zeros(o.ndofs, dtype=torch.float64)
    y = torch.zeros(o.ndofs, dtype=torch.float64, device="cuda")
    L = capi.lib()
    import ctypes
    rc = L.sem_apply(g.ctx, 1.0, 1.0, ctypes.c_void_p(u_host.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                     capi.SEM_PREC_FP64, None)
    assert rc == capi.SEM_ERR_ARG
    rc = L.sem_apply(g.ctx, 1.0, 1.0, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                     capi.SEM_PREC_FP64, None)
    assert rc == capi.SEM_ERR_ARG
    with pytest.raises(capi.SemError):
        g.cg_solve(30.0, y, y.clone(), precond=capi.SEM_PC_GMG + 5)


def test_bad_mesh_is_rejected():
    s = W.slab(2, 1, 1, (2.0, 1.0, 1.0))
    v = s.flat_vertices().copy()
    v[1, 0] = 2.5  # pull the middle bottom vertex past its right neighbour: inverted cell
    with pytest.raises(capi.SemError) as ei:
        gb.Slab(v, 2, 1, 1, 2, "LGL")
    assert ei.value.code == capi.SEM_ERR_BAD_MESH


def _oracle_run(o, tissue, dt, nsteps, region, amp, t_off, u0=None):
    md = MD.Monodomain(o, tissue, dt, region=region, amplitude=amp, t_on=0.0, t_off=t_off)
    st = MD.rest_state(o.ndofs)
    if u0 is not None:
        st = dict(u=u0.copy(), u_prev=u0.copy(), h=st["h"], h_prev=st["h_prev"], n=0)
    return md.run(st, nsteps)


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_one_step_and_first_bdf2_step(quad):
    s, tissue, g, o = _small(2, quad, perturb=0.1)
    u0 = W.uniform_vector(o.ndofs, -85.0, 20.0, seed=W.SEED_U)
    dt = 0.05
    box = (0.0, 0.0, 0.0, 1.5, 1.5, 1.5)
    g.set_ionic()
    g.set_stimulus("box", box, 50.0, 0.0, 1.0)
    st = g.new_state(torch.tensor(u0, device="cuda"), 1.0)
    for k in (1, 2):
        st.step(dt, 1, rtol=1e-13, maxit=5000)
        u, h, n = st.get()
        ref = _oracle_run(o, tissue, dt, k, ("box", box), 50.0, 1.0, u0=u0)
        assert n == k
        assert rel(u.cpu().numpy(), ref["u"]) < 1e-10
        assert rel(h.cpu().numpy(), ref["h"]) < 1e-12


@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_hundred_steps_small_slab(quad):
    """The small-slab workload: 20 x 7 x 3 mm, 8 x 4 x 2 elements, p = 2, rest
    state, 50 mV/ms corner stimulus for 1 ms, dt = 0.05 ms, 100 steps."""
    s, tissue, g, o = _small(2, quad)
    dt = 0.05
    box = (0.0, 0.0, 0.0, 1.5, 1.5, 1.5)
    g.set_ionic()
    g.set_stimulus("box", box, 50.0, 0.0, 1.0)
    st = g.new_state(-85.0, 1.0)
    stats = st.step(dt, 100, rtol=1e-13, maxit=5000)
    assert stats.steps == 100 and stats.cg_iters > 100
    u, h, n = st.get()
    ref = _oracle_run(o, tissue, dt, 100, ("box", box), 50.0, 1.0)
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-10
    assert rel(h.cpu().numpy(), ref["h"]) < 1e-10
    # the stimulus excited the corner
    assert ref["u"].max() > 0.0


def test_step_host_matches_device_step():
    s, tissue, g, o = _small(2, "LGL")
    g.set_ionic()
    g.set_stimulus("box", (0, 0, 0, 1.5, 1.5, 1.5), 50.0, 0.0, 1.0)
    st = g.new_state(-85.0, 1.0)
    st.step(0.05, 3, rtol=1e-12)
    ud, hd, _ = st.get()
    u = torch.full((o.ndofs,), -85.0, dtype=torch.float64).pin_memory()
    up = u.clone().pin_memory()
    h = torch.ones(o.ndofs, dtype=torch.float64).pin_memory()
    hp = h.clone().pin_memory()
    for n in range(3):
        capi.sem_step_host(g.ctx, u, up, h, hp, n, 0.05, 1e-12, 0.0, 1000)
    torch.cuda.synchronize()
    # the same step, up to the solver tolerance: the device run's third step takes
    # its initial residual from the second step's solve (carried), the host steps
    # apply the operator
    assert rel(u.numpy(), ud.cpu().numpy()) < 1e-11 and rel(h.numpy(), hd.cpu().numpy()) < 1e-13


@pytest.mark.parametrize("layout", ["pinned", "pageable", "pinned_offset"])
@pytest.mark.parametrize("precision", [capi.SEM_PREC_FP64, capi.SEM_PREC_DF64])
def test_step_host_out_matches_device_step(layout, precision):
    """Separate output arrays, rotated by the caller; page-locked inputs are read by
    the device in place, pageable ones are staged by copies.  The slab has an odd
    number of nodes (765): the double-float ionic update's two-node kernel does
    the last node alone; arrays that start 8 bytes past a 16-byte boundary
    (pinned_offset) take its one-node kernel."""
    s, tissue, g, o = _small(2, "LGL")
    g.set_ionic()
    g.set_stimulus("box", (0, 0, 0, 1.5, 1.5, 1.5), 50.0, 0.0, 1.0)
    capi.sem_set_operator_precision(g.ctx, precision)
    st = g.new_state(-85.0, 1.0)
    st.step(0.05, 4, rtol=1e-12)
    ud, hd, _ = st.get()

    def arr(v):
        if layout == "pinned_offset":
            t = torch.full((o.ndofs + 1,), v, dtype=torch.float64).pin_memory()[1:]
            assert t.data_ptr() % 16 == 8
            return t
        t = torch.full((o.ndofs,), v, dtype=torch.float64)
        return t.pin_memory() if layout == "pinned" else t

    us = [arr(-85.0), arr(-85.0), arr(0.0)]  # u^{n-1}, u^n, free
    hs = [arr(1.0), arr(1.0), arr(0.0)]
    for n in range(4):
        before = (us[0].clone(), us[1].clone(), hs[0].clone(), hs[1].clone())
        capi.sem_step_host_out(g.ctx, us[1], us[0], hs[1], hs[0], us[2], hs[2], n, 0.05, 1e-12, 0.0, 1000)
        # the inputs are not modified
        assert torch.equal(before[0], us[0]) and torch.equal(before[1], us[1])
        assert torch.equal(before[2], hs[0]) and torch.equal(before[3], hs[1])
        us = [us[1], us[2], us[0]]
        hs = [hs[1], hs[2], hs[0]]
    torch.cuda.synchronize()
    # up to the solver tolerance (the device run carries the initial residual from step 3 on)
    assert rel(us[1].numpy(), ud.cpu().numpy()) < 1e-11 and rel(hs[1].numpy(), hd.cpu().numpy()) < 1e-13
    # an output that overlaps an input is refused
    with pytest.raises(capi.SemError):
        capi.sem_step_host_out(g.ctx, us[1], us[0], hs[1], hs[0], us[1], hs[2], 4, 0.05, 1e-12, 0.0, 1000)


def test_activation_times_match_oracle():
    """Activation times (Eq. tau) over 60 steps of the small slab with a corner
    stimulus: max |du/dt| per node to 1e-9 of the largest, and the time wherever
    the oracle's two largest step derivatives differ by more than 1e-7."""
    from oracle import activation as ACT
    s, tissue, g, o = _small(2, "LGL")
    dt = 0.05
    box = (0.0, 0.0, 0.0, 1.5, 1.5, 1.5)
    g.set_ionic()
    g.set_stimulus("box", box, 50.0, 0.0, 1.0)
    st = g.new_state(-85.0, 1.0)
    st.track_activation(True)
    st.step(dt, 60, rtol=1e-13, maxit=5000)
    tau, dmax = st.activation()
    tau, dmax = tau.cpu().numpy(), dmax.cpu().numpy()
    md = MD.Monodomain(o, tissue, dt, region=("box", box), amplitude=50.0, t_on=0.0, t_off=1.0)
    # the oracle's derivatives at every step, for the separation test
    state = MD.rest_state(o.ndofs)
    ds = []
    for _ in range(60):
        new = md.step(state)
        ds.append(np.abs(ACT.scheme_derivative(new["u"], state["u"], state["u_prev"], new["n"], dt)))
        state = new
    ds = np.array(ds)
    tref = dt * (1 + np.argmax(ds, axis=0))
    dref = ds.max(axis=0)
    assert np.abs(dmax - dref).max() <= 1e-9 * dref.max()
    # unique maxima (the two largest step derivatives well apart, mostly the
    # activated nodes): the same step; elsewhere (resting nodes with near ties)
    # the step the GPU chose attains the oracle's maximum
    top2 = np.sort(ds, axis=0)[-2:]
    sep = (top2[1] - top2[0]) > 1e-7 * dref.max()
    assert sep.sum() >= 100
    assert np.array_equal(tau[sep], tref[sep])
    k = np.rint(tau / dt).astype(int) - 1
    assert ((k >= 0) & (k < 60)).all()
    assert (ds[k, np.arange(o.ndofs)] >= dref - 1e-9 * dref.max()).all()
    # the front moved: the far corner activates later than the stimulated one
    assert dref.max() > 10.0 and tref.max() > tref.min()
    # disabling keeps the values; re-enabling resets them
    st.track_activation(False)
    st.step(dt, 2, rtol=1e-13, maxit=5000)
    tau2, _ = st.activation()
    assert np.array_equal(tau2.cpu().numpy(), tau, equal_nan=True)
    st.track_activation(True)
    _, d3 = st.activation()
    assert (d3.cpu().numpy() == -1.0).all()
    st.close()


def test_checkpoint_restore_resumes_identically():
    s, tissue, g, o = _small(2, "LGL")
    g.set_ionic()
    g.set_stimulus("box", (0, 0, 0, 1.5, 1.5, 1.5), 50.0, 0.0, 1.0)
    st = g.new_state(-85.0, 1.0)
    st.step(0.05, 4, rtol=1e-13)
    ck = st.checkpoint()
    assert ck["n"] == 4
    st.step(0.05, 3, rtol=1e-13)
    ua, ha, na = st.get()
    st2 = g.new_state(0.0, 0.0)
    st2.restore(ck)
    st2.step(0.05, 3, rtol=1e-13)
    ub, hb, nb = st2.get()
    assert na == nb == 7
    # up to the solver tolerance: the first run's fifth step carries its initial
    # residual from the fourth, the restored state's applies the operator
    assert rel(ub.cpu().numpy(), ua.cpu().numpy()) < 1e-12


@pytest.mark.parametrize("precond", [capi.SEM_PC_JACOBI, capi.SEM_PC_GMG])
def test_carried_initial_residual(precond):
    """Consecutive time steps of one state take the initial residual of step n+1
    from step n's solve (A u^n = b_n - r_n) instead of an operator apply.  12
    steps in one call against 12 calls separated by an entry point that ends the
    carry (sem_set_deterministic): the same solution to the solver tolerance, the
    same iteration counts, and fewer kernel launches; a state restored in between
    does not inherit the carry; and both match the oracle's 12 steps."""
    s, tissue, g, o = _small(2, "LGL")
    g.set_ionic()
    box = (0.0, 0.0, 0.0, 1.5, 1.5, 1.5)
    g.set_stimulus("box", box, 50.0, 0.0, 1.0)
    capi.sem_set_operator_precision(g.ctx, gb.SEM_PREC_DF64)
    capi.sem_set_gmg(g.ctx, 3, 10, 100, capi.SEM_PREC_FP32_BF16)
    st = g.new_state(-85.0, 1.0)
    carried = st.step(0.05, 12, rtol=1e-13, maxit=2000, precond=precond)
    ua, ha, _ = st.get()
    st.close()
    st = g.new_state(-85.0, 1.0)
    launches, iters = 0, 0
    for _ in range(12):
        capi.sem_set_deterministic(g.ctx, False)  # ends the carry
        stt = st.step(0.05, 1, rtol=1e-13, maxit=2000, precond=precond)
        launches += stt.kernel_launches
        iters += stt.cg_iters
    ub, hb, _ = st.get()
    assert rel(ua.cpu().numpy(), ub.cpu().numpy()) < 1e-12
    assert abs(carried.cg_iters - iters) <= 2
    if carried.cg_iters == iters:  # then only the initial residuals differ: 10 applies fewer
        assert carried.kernel_launches < launches
    ref = _oracle_run(o, tissue, 0.05, 12, ("box", box), 50.0, 1.0)
    assert rel(ua.cpu().numpy(), ref["u"]) < 1e-10
    # a restored state (same n, same alpha) starts from a true residual
    ck = st.checkpoint()
    st2 = g.new_state(0.0, 0.0)
    st2.restore(ck)
    st.step(0.05, 1, rtol=1e-13, maxit=2000, precond=precond)
    st2.step(0.05, 1, rtol=1e-13, maxit=2000, precond=precond)
    assert rel(st.get()[0].cpu().numpy(), st2.get()[0].cpu().numpy()) < 1e-12
    st.close()
    st2.close()
    g.close()


@pytest.mark.parametrize("op", [capi.SEM_PREC_DF64, capi.SEM_PREC_FP64])
@pytest.mark.parametrize("layout", ["pinned", "pageable"])
def test_step_host_out_checked_carry(op, layout):
    """sem_step_host_out with the multigrid PCG carries the initial residual from
    one call to the next when the caller passes back the u_next it got (checked
    on the device, bit for bit): the same carried-solve counts as sem_step (none
    for the BDF1 step and the step after it, whose operator differs), the same
    solution to the solver tolerance, and the oracle's 8 steps; a u changed by the
    caller, or a call that does not continue the last one, applies the operator."""
    s, tissue, g, o = _small(2, "LGL")
    g.set_ionic()
    box = (0.0, 0.0, 0.0, 1.5, 1.5, 1.5)
    g.set_stimulus("box", box, 50.0, 0.0, 1.0)
    capi.sem_set_operator_precision(g.ctx, op)
    capi.sem_set_gmg(g.ctx, 3, 10, 100, capi.SEM_PREC_FP32_BF16)
    nsteps, dt, rtol = 8, 0.05, 1e-13
    st = g.new_state(-85.0, 1.0)
    dev = st.step(dt, nsteps, rtol=rtol, maxit=2000, precond=capi.SEM_PC_GMG)
    assert dev.carried_solves == nsteps - 2
    ud, hd, _ = st.get()
    st.close()

    def arr(v):
        t = torch.full((o.ndofs,), v, dtype=torch.float64)
        return t.pin_memory() if layout == "pinned" else t

    us = [arr(-85.0), arr(-85.0), arr(0.0)]  # u^{n-1}, u^n, free
    hs = [arr(1.0), arr(1.0), arr(0.0)]
    counts = []
    for n in range(nsteps):
        stt = capi.sem_step_host_out(g.ctx, us[1], us[0], hs[1], hs[0], us[2], hs[2], n, dt, rtol, 0.0, 2000,
                                     capi.SEM_PC_GMG)
        counts.append(stt.carried_solves)
        us = [us[1], us[2], us[0]]
        hs = [hs[1], hs[2], hs[0]]
    assert counts == [0, 0] + [1] * (nsteps - 2), counts
    assert rel(us[1].numpy(), ud.cpu().numpy()) < 1e-11 and rel(hs[1].numpy(), hd.cpu().numpy()) < 1e-13
    ref = _oracle_run(o, tissue, dt, nsteps, ("box", box), 50.0, 1.0)
    assert rel(us[1].numpy(), ref["u"]) < 1e-10

    def step_from(u, u_prev, h, h_prev, n):
        un, hn = arr(0.0), arr(0.0)
        stt = capi.sem_step_host_out(g.ctx, u, u_prev, h, h_prev, un, hn, n, dt, rtol, 0.0, 2000,
                                     capi.SEM_PC_GMG)
        return stt.carried_solves, un, hn

    # u changed by the caller in one entry: the operator is applied
    u_mod = us[1].clone()
    u_mod[o.ndofs // 2] += 1e-3
    u_mod = u_mod.pin_memory() if layout == "pinned" else u_mod
    c, un, hn = step_from(u_mod, us[0], hs[1], hs[0], nsteps)
    assert c == 0
    # the same n again does not continue the last call: no carry, the same result
    c2, un2, hn2 = step_from(u_mod, us[0], hs[1], hs[0], nsteps)
    assert c2 == 0 and rel(un2.numpy(), un.numpy()) < 1e-12
    # continuing from what that call returned carries again
    un2 = un2.pin_memory() if layout == "pinned" else un2
    hn2 = hn2.pin_memory() if layout == "pinned" else hn2
    c3, _, _ = step_from(un2, u_mod, hn2, hs[1], nsteps + 1)
    assert c3 == 1
    # the step from the changed u agrees with the same step of a state set from those arrays
    st = g.new_state(0.0, 0.0)
    st.restore(dict(u=u_mod.cuda(), u_prev=us[0].cuda(), h=hs[1].cuda(), h_prev=hs[0].cuda(), n=nsteps))
    st.step(dt, 1, rtol=rtol, maxit=2000, precond=capi.SEM_PC_GMG)
    ur, hr, _ = st.get()
    st.close()
    assert rel(un.numpy(), ur.cpu().numpy()) < 1e-11 and rel(hn.numpy(), hr.cpu().numpy()) < 1e-13
    g.close()


def test_timing_samples_one_solve_in_ten():
    """With timing on, the multigrid PCG times the outer apply and the fine-level
    residual apply in the first iteration of one solve in ten (the first after
    enabling, then every tenth), the Jacobi CG the apply of that iteration; with
    timing off nothing is timed."""
    s, tissue, g, o = _small(2, "LGL")
    g.set_ionic()
    g.set_stimulus("box", (0.0, 0.0, 0.0, 1.5, 1.5, 1.5), 50.0, 0.0, 2.0)  # every step iterates
    capi.sem_set_operator_precision(g.ctx, gb.SEM_PREC_DF64)
    capi.sem_set_gmg(g.ctx, 3, 10, 100, capi.SEM_PREC_FP32_BF16)
    st = g.new_state(-85.0, 1.0)
    off = st.step(0.05, 5, rtol=1e-12, maxit=200, precond=capi.SEM_PC_GMG)
    assert off.cg_iters >= 5
    assert off.n_apply == 0 and off.n_smoother_apply == 0
    g.set_timing(True)
    on = st.step(0.05, 20, rtol=1e-12, maxit=200, precond=capi.SEM_PC_GMG)
    assert on.cg_iters >= 20
    assert on.n_apply == 2 and on.n_smoother_apply == 2, (on.n_apply, on.n_smoother_apply)
    assert on.apply_ms > 0.0 and on.smoother_apply_ms > 0.0
    g.set_timing(True)  # restarts the count: the Jacobi CG samples its first apply the same way
    jac = st.step(0.05, 20, rtol=1e-12, maxit=2000, precond=capi.SEM_PC_JACOBI)
    assert jac.n_apply == 2 and jac.n_smoother_apply == 0 and jac.apply_ms > 0.0, (jac.n_apply, jac.apply_ms)
    g.set_timing(False)
    st.close()
    g.close()


def test_ionic_parameters_reach_the_kernel():
    prm = dict(ionic.DEFAULT_PARAMS)
    prm["tau_out"] = 3.0
    s, tissue, g, o = _small(1, "LGL", dims=(2, 2, 1))
    g.set_ionic(**prm)
    st = g.new_state(-60.0, 0.8)
    st.step(0.05, 5, rtol=1e-13)
    u, h, _ = st.get()
    ref = ionic.single_cell_semi_implicit(-60.0, 0.8, 0.25, 0.05, prm)
    assert np.abs(u.cpu().numpy() - ref[0]).max() < 1e-10 * abs(ref[0])


@pytest.mark.parametrize("precond", [capi.SEM_PC_JACOBI, capi.SEM_PC_GMG])
@pytest.mark.parametrize("quad", ["LGL", "LG"])
def test_df64_operator_in_cg_and_time_steps(quad, precond):
    """The double-float operator inside CG (and the multigrid PCG) reaches the
    FP64 solution, and 20 time steps match the oracle to 1e-10."""
    s, tissue, g, o = _small(3, quad, perturb=0.1, dims=(4, 3, 2))
    capi.sem_set_operator_precision(g.ctx, capi.SEM_PREC_DF64)
    capi.sem_set_gmg(g.ctx, 3, 10, 50, capi.SEM_PREC_FP32)
    alpha = 1.5 / 0.05
    A = Mh.assemble(o, tissue, alpha, 1.0)
    b = W.uniform_vector(o.ndofs, -1.0, 1.0, seed=3)
    import scipy.sparse.linalg as spla
    xref = spla.spsolve(A.tocsc(), b)
    x = torch.zeros(o.ndofs, dtype=torch.float64, device="cuda")
    g.cg_solve(alpha, torch.tensor(b, device="cuda"), x, rtol=1e-13, maxit=5000, precond=precond)
    assert rel(x.cpu().numpy(), xref) < 1e-11
    box = (0.0, 0.0, 0.0, 3.0, 3.0, 1.5)
    g.set_ionic()
    g.set_stimulus("box", box, 50.0, 0.0, 1.0)
    st = g.new_state(-85.0, 1.0)
    st.step(0.05, 20, rtol=1e-13, maxit=5000, precond=precond)
    u, _, _ = st.get()
    ref = _oracle_run(o, tissue, 0.05, 20, ("box", box), 50.0, 1.0)
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-10


def test_benchmark_time_step_full_size():
    """The benchmarked mixed-precision time step on its full-size workload
    (83 x 29 x 13 perturbed Q4 elements, 2,064,933 DOFs, SEM-NI, rotating
    fibres, sphere stimulus): flexible FP64 PCG with the double-float operator,
    bf16-metric V-cycle with Chebyshev(6) and Chebyshev(5) on the coarsest
    level, the first of at most 300,000 nodes, rtol 1e-10.  After 20 steps (the
    stimulus has just ended)
    one more step is checked:
      - the gate update at every node against the oracle's BDF2 gate (Eq.
        ionic_discr);
      - the FP64 residual of the solved system (Eq. linsys) over all nodes, with
        b from the oracle's right-hand side (Eq. matrix_rhs) and the mass
        diagonal, and A u from the FP64 apply, whose rows at this size are
        pinned to the oracle by test_sweep_workload_sampled_rows;
      - the solution against the plain FP64 path's (FP64 operator, Jacobi-CG)
        from the same state."""
    dt, rtol = 0.05, 1e-10
    s = W.sweep_slab(4)
    ne = s.n_elements
    tissue = (np.full(ne, 0.12), np.full(ne, 0.03), W.transmural_fiber_angles(s))
    centre = W.seeded_point(s.lengths, 1.5, seed=W.SEED_STIM)
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, 4, "LGL")
    g.set_tissue(*tissue)
    g.set_ionic()
    g.set_stimulus("sphere", (*centre, 1.5), 50.0, 0.0, 1.0)
    capi.sem_set_gmg(g.ctx, 6, 5, 300000, gb.SEM_PREC_FP32_BF16)
    capi.sem_set_operator_precision(g.ctx, gb.SEM_PREC_DF64)
    st = g.new_state(-85.0, 1.0)
    st.step(dt, 20, rtol=rtol, maxit=2000, precond=gb.SEM_PC_GMG)
    ck = st.checkpoint()
    assert ck["n"] == 20
    st.step(dt, 1, rtol=rtol, maxit=2000, precond=gb.SEM_PC_GMG)  # t = 1.05 ms: no stimulus
    u1, h1, n1 = st.get()
    assert n1 == 21
    un, unm1, hn, hnm1 = (ck[k].cpu().numpy() for k in ("u", "u_prev", "h", "h_prev"))
    assert un.max() > -40.0  # the stimulated region has depolarised: the step is nonlinear

    prm = ionic.DEFAULT_PARAMS
    us = 2.0 * un - unm1
    h_ref = ionic.gate_bdf2(hn, hnm1, us, dt, prm)
    assert np.abs(h1.cpu().numpy() - h_ref).max() < 1e-13

    alpha = 1.5 / dt
    mdiag = g.diagonal(1.0, 0.0).cpu().numpy()
    b = mdiag * ((4.0 * un - unm1) / (2.0 * dt) - ionic.i_ion(us, h_ref, prm))
    r = b - g.apply(u1, alpha, 1.0).cpu().numpy()
    assert np.linalg.norm(r) <= 2.0 * rtol * np.linalg.norm(b)

    capi.sem_set_operator_precision(g.ctx, gb.SEM_PREC_FP64)
    st64 = g.new_state(-85.0, 1.0)
    st64.restore(ck)
    st64.step(dt, 1, rtol=rtol, maxit=2000, precond=gb.SEM_PC_JACOBI)
    u64, _, _ = st64.get()
    assert rel(u1.cpu().numpy(), u64.cpu().numpy()) < 1e-8
    st64.close()
    st.close()
    g.close()
    torch.cuda.empty_cache()


def test_mixed_precision_30m_matches_fp64_multigrid():
    """The ~30 M DOF mixed-precision workload at p = 4 (207 x 72 x 31 perturbed Q4
    elements, 29,947,625 DOFs, SEM-NI, rotating fibres, sphere stimulus): three time
    steps (BDF1, then BDF2) of the mixed solver -- flexible FP64 PCG with the
    double-float operator and the bf16-metric V-cycle, Chebyshev(6) on every level,
    coarsening down to 300,000 nodes -- against three steps of flexible PCG with the
    FP64 operator and an all-FP64 V-cycle on the same hierarchy, both at rtol 1e-10
    from the rest state: u and h agree to 1e-8 relative in the 2-norm and the max
    norm.  The FP64 operator at this size is pinned to the oracle by sampled rows."""
    dt, rtol, nsteps = 0.05, 1e-10, 3
    s = W.slab(207, 72, 31, (20.0, 7.0, 3.0), perturb=0.1, seed=W.SEED_MESH)
    ne = s.n_elements
    tissue = (np.full(ne, 0.12), np.full(ne, 0.03), W.transmural_fiber_angles(s))
    centre = W.seeded_point(s.lengths, 1.5, seed=W.SEED_STIM)
    g = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, 4, "LGL")
    assert g.ndofs == 829 * 289 * 125  # 29,947,625
    g.set_tissue(*tissue)
    g.set_ionic()
    g.set_stimulus("sphere", (*centre, 1.5), 50.0, 0.0, 1.0)

    o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, 4, "LGL")
    uvec = W.uniform_vector(g.ndofs, seed=W.SEED_U)
    y = g.apply(torch.tensor(uvec, device="cuda"), 1.5 / dt, 1.0)
    idx = W.seeded_indices(g.ndofs, 12, seed=7)
    ref = Mh.sampled_rows(o, tissue, uvec, idx, 1.5 / dt, 1.0)
    yi = y[torch.tensor(idx, device="cuda")].cpu().numpy()
    assert np.abs(yi - ref).max() < 1e-12 * np.abs(ref).max()
    del y

    out = {}
    for name, op, prec in (("fp64", gb.SEM_PREC_FP64, gb.SEM_PREC_FP64),
                           ("mixed", gb.SEM_PREC_DF64, gb.SEM_PREC_FP32_BF16)):
        capi.sem_set_operator_precision(g.ctx, op)
        capi.sem_set_gmg(g.ctx, 6, 6, 300000, prec)
        st = g.new_state(-85.0, 1.0)
        st.step(dt, nsteps, rtol=rtol, maxit=8000, precond=gb.SEM_PC_GMG)
        u, h, n = st.get()
        assert n == nsteps
        out[name] = (u.clone(), h.clone())
        st.close()
    (u64, h64), (umx, hmx) = out["fp64"], out["mixed"]
    assert float(umx.max()) > -85.0 + 1.0  # the stimulus has moved u
    assert float(torch.linalg.norm(umx - u64) / torch.linalg.norm(u64)) < 1e-8
    assert float((umx - u64).abs().max() / u64.abs().max()) < 1e-8
    assert float(torch.linalg.norm(hmx - h64) / torch.linalg.norm(h64)) < 1e-8
    assert float((hmx - h64).abs().max() / h64.abs().max()) < 1e-8
    g.close()
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("first", [True, False])
def test_double_float_ionic_update_matches_fp64(first):
    """The ionic update and right-hand side in double-float arithmetic (used with
    the double-float operator) against the FP64 kernel, from a state whose u
    spans -90..40 mV (the gate's exponent from -112, where it underflows, to 18)
    and h spans 0..1: one step (BDF1 from n = 0, else BDF2), Jacobi-CG at rtol
    1e-13; the new gate agrees to 1e-13 absolute and u to 1e-11 relative, and the
    gate matches the oracle's closed-form BDF update at every node."""
    s, tissue, g, o = _small(3, "LGL", perturb=0.1, dims=(6, 4, 3))
    g.set_ionic()
    g.set_stimulus("box", (0.0, 0.0, 0.0, 5.0, 3.0, 1.5), 50.0, 0.0, 1.0)
    n = g.ndofs
    u = torch.tensor(W.uniform_vector(n, -90.0, 40.0, seed=31), device="cuda")
    um = torch.tensor(W.uniform_vector(n, -90.0, 40.0, seed=32), device="cuda")
    h = torch.tensor(W.uniform_vector(n, 0.0, 1.0, seed=33), device="cuda")
    hm = torch.tensor(W.uniform_vector(n, 0.0, 1.0, seed=34), device="cuda")
    state = {"u": u, "u_prev": um, "h": h, "h_prev": hm, "n": 0 if first else 5}
    res = {}
    for prec in (gb.SEM_PREC_FP64, gb.SEM_PREC_DF64):
        capi.sem_set_operator_precision(g.ctx, prec)
        st = g.new_state(-85.0, 1.0)
        st.restore(state)
        st.step(0.05, 1, rtol=1e-13, maxit=5000, precond=capi.SEM_PC_JACOBI)
        u1, h1, _ = st.get()
        res[prec] = (u1.cpu().numpy(), h1.cpu().numpy())
        st.close()
    (u64, h64), (udf, hdf) = res[gb.SEM_PREC_FP64], res[gb.SEM_PREC_DF64]
    assert np.abs(hdf - h64).max() < 1e-13
    assert rel(udf, u64) < 1e-11
    prm = ionic.DEFAULT_PARAMS
    un, unm1, hn, hnm1 = (state[k].cpu().numpy() for k in ("u", "u_prev", "h", "h_prev"))
    if first:
        h_ref = ionic.gate_bdf1(hn, un, 0.05, prm)
    else:
        h_ref = ionic.gate_bdf2(hn, hnm1, 2.0 * un - unm1, 0.05, prm)
    assert np.abs(hdf - h_ref).max() < 1e-13
    g.close()
