"""GPU calibration parity: pm_fit / batched plan / autograd kernels / pm_predict
vs the FP64 oracle (scipy leastsq, column-scaled least squares, symbolic
derivatives).  Parameter agreement is measured as max_i |p_i - p_i*| / |p_i*|."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import pm_inputs  # noqa: E402
import paper_1904_09538_gb300 as pm  # noqa: E402
from paper_1904_09538_gb300 import autograd as pag  # noqa: E402
from oracle import fit as ofit  # noqa: E402
from oracle.model import Model as OModel, overlap_expr  # noqa: E402
from oracle.features import features as ofeatures, feature_value as ofeature_value  # noqa: E402
from oracle.quasipoly import extrapolate  # noqa: E402

PTOL = 1e-6


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def perr(p, ref):
    """max_i |p_i - ref_i| / |ref_i| (parameters carry different units)."""
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(np.asarray(p) - ref) / np.abs(ref)))


LIN = ("p_launch * f_sync_kernel_launch + p_group * f_thread_groups + p_add * f_op_float32_add + "
       "p_madd * f_op_float32_madd + p_gmem * f_mem_access_global_float32 + p_lmem * f_mem_access_local_float32")
OVL = overlap_expr("p_launch * f_sync_kernel_launch + p_group * f_thread_groups",
                   "p_gmem * f_mem_access_global_float32",
                   "p_madd * f_op_float32_madd + p_lmem * f_mem_access_local_float32")


def design(l, seed, nf=6):
    """Feature rows: launch = 1, work-groups in [1e2, 1e4], counts in [1e5, 1e7]."""
    X = pm_inputs.integers((l, nf), seed, 10 ** 5, 10 ** 7).astype(np.float64)
    X[:, 0] = 1.0
    X[:, 1] = pm_inputs.integers((l,), seed + 1000, 100, 10 ** 4)
    return X


def synth(expr, X, p_true, sigma, seed):
    """Outputs of the model at p_true (a name -> value dict), with relative noise."""
    om = OModel("f_wall_time", expr)
    F = [dict(zip(om.features, row)) for row in X]
    t = np.array([om.eval(p_true, f) for f in F])
    return t * (1 + sigma * pm_inputs.noise((len(t),), seed)), om, F


def oracle_row(om, kernel, var, target, period, degree, start, **params):
    """A design-matrix row from the oracle's own counts: each model feature
    on kernel(params, var = target), by brute-force enumeration at small
    sizes of target's residue class and exact quasi-polynomial
    extrapolation, so that no oracle input comes from the library."""
    cache = {}

    def col(i):
        def f(v):
            if v not in cache:
                recs = ofeatures(kernel, **dict(params, **{var: v}))
                cache[v] = [ofeature_value(name, recs) for name in om.features]
            return cache[v][i]
        return f
    return np.array([float(extrapolate(col(i), target, period, degree, start)) for i in range(len(om.features))])


def vec(model, pd):
    return np.array([pd[n] for n in model.params])


P_LIN = dict(p_launch=5e-6, p_group=2e-9, p_add=4e-12, p_madd=3e-12, p_gmem=6e-12, p_lmem=2e-12)
P_OVL = dict(p_launch=5e-6, p_group=2e-9, p_gmem=6e-12, p_madd=3e-12, p_lmem=2e-12, p_edge=3e4)


@pytest.mark.parametrize("sigma", [0.0, 1e-3, 1e-2])
def test_linear_fit_vs_oracle(sigma):
    dev()
    X = design(120, 3)
    t, om, F = synth(LIN, X, P_LIN, sigma, 4)
    m = pm.Model("f_wall_time", LIN)
    assert m.is_linear and m.features == om.features
    p, rep = m.fit(X, t)
    po, info = ofit.fit(om, F, t)
    assert rep["status"] == 0 and rep["linear"] and rep["rank"] == 6
    assert perr(p, po) <= PTOL, perr(p, po)
    if sigma == 0:
        assert perr(p, vec(om, P_LIN)) <= PTOL


def test_rank_deficient_matmul_design():
    # flops, global, local, work-groups on the PF matmul at n = 256..768 are
    # rank 2 (all columns in span{n^3, n^2}); predictions at n = 896 are unique
    dev()
    expr = ("p_f * f_op_float32_madd + p_g * f_mem_access_global_float32 + p_s * f_mem_access_local_float32 + "
            "p_l * f_thread_groups")
    m = pm.Model("f_wall_time", expr)
    om = OModel("f_wall_time", expr)
    ns = [256, 384, 512, 640, 768]
    X = np.array([oracle_row(om, "mm_pf", "n", n, 16, 3, 16) for n in ns])
    t = np.array([1e-12 * n ** 3 + 3e-10 * n ** 2 for n in ns])
    p, rep = m.fit(X, t)
    po, info = ofit.fit(om, [dict(zip(om.features, r)) for r in X], t)
    assert info["rank_deficient"] and rep["status"] == -5 and rep["rank"] == info["rank"] == 2
    x896 = oracle_row(om, "mm_pf", "n", 896, 16, 3, 16)
    pred = m.predict(p, x896[None, :])[0]
    pred_o = float(x896 @ po)
    assert abs(pred / pred_o - 1) <= 1e-6
    assert perr(p, po) <= 1e-5  # min-norm solutions in the same column-scaled coordinates


@pytest.mark.parametrize("sigma,seed", [(0.0, 5), (1e-3, 6), (1e-2, 7)])
def test_overlap_fit_vs_oracle(sigma, seed):
    dev()
    X = design(200, seed, nf=5)
    t, om, F = synth(OVL, X, P_OVL, sigma, seed + 100)
    m = pm.Model("f_wall_time", OVL)
    assert not m.is_linear
    p0 = vec(om, P_OVL) * (1 + 0.3 * pm_inputs.uniform((6,), seed, dtype=np.float64))
    p, rep = m.fit(X, t, p0=p0)
    po, info = ofit.fit(om, F, t, p0=p0)
    assert rep["status"] == 0, rep
    assert perr(p, po) <= PTOL, (perr(p, po), p, po)


def test_overlap_fit_default_start_point():
    dev()
    X = design(150, 9, nf=5)
    t, om, F = synth(OVL, X, P_OVL, 1e-3, 10)
    m = pm.Model("f_wall_time", OVL)
    p, rep = m.fit(X, t)
    po, _ = ofit.fit(om, F, t)
    pred = m.predict(p, X)
    pred_o = ofit.predict(om, po, F)
    assert np.max(np.abs(pred / pred_o - 1)) <= 1e-5


def test_batched_uneven_matches_single_and_oracle():
    dev()
    K = 12
    ls = pm_inputs.row_counts(K, 42)
    models, Xs, ts, p0s, refs = [], [], [], [], []
    for k in range(K):
        expr = LIN if k % 2 == 0 else OVL
        nf = 6 if k % 2 == 0 else 5
        ptrue = P_LIN if k % 2 == 0 else P_OVL
        X = design(int(ls[k]), 200 + k, nf=nf)
        t, om, F = synth(expr, X, ptrue, 1e-2, 300 + k)
        p0 = vec(om, ptrue) * 1.2
        models.append(pm.Model("f_wall_time", expr))
        Xs.append(X)
        ts.append(t)
        p0s.append(p0)
        refs.append(ofit.fit(om, F, t, p0=p0)[0])
    for threads in (64, 128, 256, 512):
        ps, reps = pm.fit_batched(models, Xs, ts, p0s, threads=threads)
        for k in range(K):
            assert reps[k]["status"] == 0, (k, reps[k])
            assert perr(ps[k], refs[k]) <= PTOL, (k, perr(ps[k], refs[k]))
    single, _ = models[1].fit(Xs[1], ts[1], p0=p0s[1])
    ps, _ = pm.fit_batched(models, Xs, ts, p0s, threads=128)
    assert np.array_equal(single, ps[1])


def test_autograd_residual_gradient_and_jacobian():
    d = dev()
    X = design(64, 51, nf=5)
    t, om, F = synth(OVL, X, P_OVL, 1e-2, 52)
    m = pm.Model("f_wall_time", OVL)
    p = vec(om, P_OVL) * 1.1
    Xd = torch.from_numpy(X).to(d)
    td = torch.from_numpy(t).to(d)
    pd = torch.from_numpy(p).to(d).requires_grad_(True)
    r = pag.Residual.apply(pd, m, Xd, td)
    r_or, J_or = ofit.residual_and_jacobian(om, F, t)
    # float-float evaluation (about 48 bits): r = 1 - g/t within 1e-13
    assert np.max(np.abs(r.detach().cpu().numpy() - r_or(p))) <= 1e-13
    rbar = pm_inputs.normal((64,), 53).astype(np.float64)
    (g,) = torch.autograd.grad(r, pd, grad_outputs=torch.from_numpy(rbar).to(d))
    J = J_or(p)
    want = J.T @ rbar
    scale = np.abs(J).T @ np.abs(rbar)
    # float-float reverse sweep: J^T rbar within 1e-11 of the sum of |terms|
    assert np.all(np.abs(g.cpu().numpy() - want) <= 1e-11 * scale)
    # Jacobian vs FP64 central differences, h = 1e-3 in scaled coordinates q = p / |p|
    Jg = pag.jacobian(m, Xd, td, pd.detach()).cpu().numpy()
    for i in range(len(p)):
        h = 1e-3 * abs(p[i])
        pp, pm_ = p.copy(), p.copy()
        pp[i] += h
        pm_[i] -= h
        fd = (r_or(pp) - r_or(pm_)) / (2 * h)
        assert np.all(np.abs(Jg[:, i] - fd) <= 1e-4 * (np.abs(fd).max() + 1e-30)), i
    # the torch.autograd gradcheck-style consistency: backward == J^T rbar
    assert np.allclose(g.cpu().numpy(), Jg.T.astype(np.float64) @ rbar, rtol=1e-4, atol=1e-4 * scale.max())


def test_jacobian_where_tanh_is_nearly_saturated():
    # global cost far below the on-chip cost: p_edge (c_gmem - c_on-chip) -8 at
    # the median row (-1 to -14 over the rows), tanh there within 1e-6 of -1.  The derivative of tanh must not
    # come from 1 - t*t of the rounded t (13 % off there): the columns of the
    # FP32 Jacobians (the LM's and the autograd kernels') match the oracle's
    # FP64 analytic Jacobian
    d = dev()
    X = design(64, 61, nf=5)
    om = OModel("f_wall_time", OVL)
    F = [dict(zip(om.features, row)) for row in X]
    P = dict(P_OVL, p_gmem=1e-14)
    cg = np.array([OModel("t", "p_gmem * f_mem_access_global_float32").eval(P, f) for f in F])
    co = np.array([OModel("t", "p_madd * f_op_float32_madd + p_lmem * f_mem_access_local_float32").eval(P, f)
                   for f in F])
    P["p_edge"] = 8.0 / float(np.median(co - cg))
    arg = P["p_edge"] * (cg - co)
    assert np.median(arg) == pytest.approx(-8.0) and np.mean(arg < -4) > 0.5
    t = np.array([om.eval(P, f) for f in F]) * (1 + 1e-2 * pm_inputs.noise((64,), 62))
    m = pm.Model("f_wall_time", OVL)
    p = vec(om, P)
    _, J_or = ofit.residual_and_jacobian(om, F, t)
    J = J_or(p)
    Jg = pag.jacobian(m, torch.from_numpy(X).to(d), torch.from_numpy(t).to(d), torch.from_numpy(p).to(d)).cpu().numpy()
    # the forward values are float-float, so even tanh + 1 (about 2e-7 here,
    # the factor of f_gmem in p_gmem's column) keeps its leading digits; the
    # FP32 reverse sweep then leaves each column within 1e-4
    for i, name in enumerate(om.params):
        assert np.all(np.abs(Jg[:, i] - J[:, i]) <= 1e-4 * np.abs(J[:, i]).max()), name
    # the LM (float-float forward values) from a start 30 % off reaches the oracle's optimum
    p0 = p * (1 + 0.3 * pm_inputs.uniform((len(p),), 63, dtype=np.float64))
    pf, rep = m.fit(X, t, p0=p0)
    po, _ = ofit.fit(om, F, t, p0=p0)
    assert rep["status"] == 0
    assert np.max(np.abs(m.predict(pf, X) / np.asarray(ofit.predict(om, po, F)) - 1)) <= 1e-5


def test_autograd_lm_matches_oracle():
    # the plain per-model LM (autograd.Function for J^T r, library step and
    # update calls) reaches the oracle's optimum within the 1e-6 bar
    d = dev()
    X = design(150, 61, nf=5)
    t, om, F = synth(OVL, X, P_OVL, 1e-2, 62)
    m = pm.Model("f_wall_time", OVL)
    p0 = vec(om, P_OVL) * 1.25
    Xd = torch.from_numpy(X).to(d)
    td = torch.from_numpy(t).to(d)
    p, rep = pag.lm_fit(m, Xd, td, p0)
    po, _ = ofit.fit(om, F, t, p0=p0)
    assert rep["status"] == 0 and 0 < rep["iterations"] < 200, rep
    assert perr(p, po) <= PTOL, perr(p, po)
    # the same fit on the batched path lands on the same point
    pb, _ = pm.fit_batched([m], [X], [t], [p0])
    assert perr(p, pb[0]) <= PTOL


def test_autograd_lm_iteration_limit_and_bad_start():
    # max_iter = 0 returns the start point with PM_ENOTCONV; a NaN start
    # point is refused before anything runs
    d = dev()
    X = design(60, 63, nf=5)
    t, om, F = synth(OVL, X, P_OVL, 1e-2, 64)
    m = pm.Model("f_wall_time", OVL)
    p0 = vec(om, P_OVL) * 1.25
    Xd, td = torch.from_numpy(X).to(d), torch.from_numpy(t).to(d)
    p, rep = pag.lm_fit(m, Xd, td, p0, max_iter=0)
    assert rep["status"] == -4 and rep["iterations"] == 0 and np.array_equal(p, p0)
    p, rep = pag.lm_fit(m, Xd, td, p0, max_iter=2)
    assert rep["status"] == -4 and rep["iterations"] == 2
    bad = p0.copy()
    bad[2] = np.nan
    with pytest.raises(pm.PMError) as e:
        pag.lm_fit(m, Xd, td, bad)
    assert e.value.status == -1


def test_predict_fp64():
    dev()
    X = design(50, 71, nf=5)
    m = pm.Model("f_wall_time", OVL)
    om = OModel("f_wall_time", OVL)
    p = vec(om, P_OVL)
    got = m.predict(p, X)
    want = ofit.predict(om, p, [dict(zip(om.features, r)) for r in X])
    assert np.max(np.abs(got / want - 1)) <= 1e-13


def test_fit_rejects_bad_data():
    dev()
    m = pm.Model("f_wall_time", LIN)
    X = design(20, 81)
    t = np.ones(20)
    t[3] = -1.0
    with pytest.raises(pm.PMError):
        m.fit(X, t)
    t[3] = np.nan
    with pytest.raises(pm.PMError):
        m.fit(X, t)


def test_fit_rejects_empty_data():
    dev()
    m = pm.Model("f_wall_time", LIN)
    with pytest.raises(pm.PMError):
        m.fit(np.zeros((0, 6)), np.zeros(0))


def test_fewer_rows_than_parameters_interpolates_with_min_norm():
    # l = 3 < m = 6: rank-deficient, the minimum-norm solution reproduces every row
    dev()
    X = design(3, 131)
    t, om, F = synth(LIN, X, P_LIN, 0.0, 132)
    m = pm.Model("f_wall_time", LIN)
    p, rep = m.fit(X, t)
    assert rep["status"] == -5 and rep["rank"] == 3
    assert np.max(np.abs(m.predict(p, X) / t - 1)) <= 1e-9
    po, _ = ofit.fit(om, F, t)      # the oracle's minimum-norm solution in the same coordinates
    assert np.max(np.abs(m.predict(po, X) / t - 1)) <= 1e-9


def test_batched_single_row_and_single_parameter_models():
    dev()
    one = pm.Model("f_wall_time", "p_madd * f_op_float32_madd")
    lin = pm.Model("f_wall_time", LIN)
    X1 = np.array([[4.0e6]])
    t1 = np.array([1.2e-5])
    X2 = design(40, 141)
    t2, _, _ = synth(LIN, X2, P_LIN, 0.0, 142)
    plan = pm.FitPlan([one, lin], [1, 40])
    p, reps = plan.run(np.concatenate([X1.ravel(), X2.ravel()]), np.concatenate([t1, t2]))
    assert reps[0]["status"] == 0 and abs(p[0] * 4.0e6 / 1.2e-5 - 1) <= 1e-12
    assert reps[1]["status"] == 0 and perr(p[1:], vec(lin, P_LIN)) <= 1e-8


OVL_BIG = overlap_expr(
    "p_launch * f_sync_kernel_launch + p_group * f_thread_groups + p_bar * f_sync_barrier_local",
    "p_g1 * f_mem_access_global_float32 + p_g2 * f_mem_access_global_float64",
    "p_madd * f_op_float32_madd + p_add * f_op_float32_add + p_lmem * f_mem_access_local_float32")
P_BIG = dict(p_launch=5e-6, p_group=2e-9, p_bar=1e-10, p_g1=6e-12, p_g2=9e-12, p_madd=3e-12, p_add=2e-12,
             p_lmem=2e-12, p_edge=3e4)


@pytest.mark.parametrize("threads", [128, 512])
@pytest.mark.parametrize("sigma,seed", [(1e-2, 31), (3e-2, 32)])
def test_large_overlap_model_converges(sigma, seed, threads):
    # nine parameters, noisy outputs, a start point 0-30 % off the generating
    # parameters: the LM must stop on its own criteria (status 0, not the
    # iteration limit) at the oracle's optimum from the same start
    dev()
    X = design(300, seed, nf=8)
    t, om, F = synth(OVL_BIG, X, P_BIG, sigma, seed + 100)
    m = pm.Model("f_wall_time", OVL_BIG)
    assert m.features == om.features and len(m.params) == 9
    p0 = vec(om, P_BIG) * (1 + 0.3 * pm_inputs.uniform((9,), seed, dtype=np.float64))
    ps, reps = pm.fit_batched([m], [X], [t], [p0], threads=threads)
    assert reps[0]["status"] == 0 and reps[0]["iterations"] < 200, reps[0]
    po, _ = ofit.fit(om, F, t, p0=p0)
    pred = m.predict(ps[0], X)
    pred_o = ofit.predict(om, po, F)
    assert np.max(np.abs(pred / pred_o - 1)) <= 1e-5


@pytest.mark.parametrize("sigma,seed", [(1e-2, 31), (3e-2, 32)])
def test_large_overlap_model_default_start(sigma, seed):
    # the same nine-parameter problems from the default start point, where
    # three coefficients of the start's linear fit come out negative and are
    # replaced by 1e-3 sum(t) / sum |their column|: both fits stop at the
    # same optimum
    dev()
    X = design(300, seed, nf=8)
    t, om, F = synth(OVL_BIG, X, P_BIG, sigma, seed + 100)
    m = pm.Model("f_wall_time", OVL_BIG)
    p, rep = m.fit(X, t)
    assert rep["status"] == 0 and rep["iterations"] < 200, rep
    po, info = ofit.fit(om, F, t)
    pred = m.predict(p, X)
    pred_o = ofit.predict(om, po, F)
    assert np.max(np.abs(pred / pred_o - 1)) <= 1e-5
    assert rep["residual"] ** 2 <= info["residual"] ** 2 * (1 + 1e-6)


def test_injected_allocation_failures_return_enomem():
    # pm_test_fail_allocation makes the n-th next allocation fail on the host
    # (no GPU fault): each entry point that allocates reports PM_ENOMEM,
    # releases what it had, and works again once the hook is disarmed
    dev()
    L = pm.lib()
    m = pm.Model("f_wall_time", LIN)
    X = design(40, 71)
    t, _, _ = synth(LIN, X, P_LIN, 0.0, 72)
    try:
        for n in (1, 4, 9):              # a fit plan allocates 12 staging buffers
            assert L.pm_test_fail_allocation(n) == 0
            with pytest.raises(pm.PMError) as ei:
                pm.FitPlan([m], [len(t)])
            assert ei.value.status == -2, ei.value
        assert L.pm_test_fail_allocation(2) == 0
        with pytest.raises(pm.PMError) as ei:
            m.predict(vec(OModel("f_wall_time", LIN), P_LIN), X)
        assert ei.value.status == -2
        host = [np.ones(1 << 16, dtype=np.float32) for _ in range(2)]
        assert L.pm_test_fail_allocation(1) == 0
        with pytest.raises(pm.PMError) as ei:
            pm.run_host("stream", host, warmup=0, trials=1, N=1 << 16)
        assert ei.value.status == -2
        assert L.pm_test_fail_allocation(-1) == -1
    finally:
        L.pm_test_fail_allocation(0)
    p, rep = m.fit(X, t)
    assert rep["status"] == 0 and perr(p, vec(OModel("f_wall_time", LIN), P_LIN)) <= PTOL
    out = pm.run_host("stream", host, warmup=0, trials=1, N=1 << 16)
    assert out["n_trials"] == 1 and np.array_equal(host[1], host[0])


def test_fit_report_condition_estimate():
    # (max/min Cholesky pivot)^2 of the unit-diagonal normal matrix: a lower
    # bound of its 2-norm condition number, within a small factor of it here;
    # +inf for the rank-deficient matmul design
    dev()
    X = design(120, 81)
    t, om, F = synth(LIN, X, P_LIN, 1e-3, 82)
    m = pm.Model("f_wall_time", LIN)
    p, rep = m.fit(X, t)
    A = X / t[:, None]
    N = A.T @ A
    d = np.sqrt(np.diag(N))
    kappa = np.linalg.cond(N / np.outer(d, d))
    assert 1.0 <= rep["cond"] <= kappa * (1 + 1e-6) and rep["cond"] >= kappa / 100, (rep["cond"], kappa)
    ps, reps = pm.fit_batched([pm.Model("f_wall_time", OVL)], [design(150, 83, nf=5)],
                              [synth(OVL, design(150, 83, nf=5), P_OVL, 1e-3, 84)[0]], threads=128)
    assert np.isfinite(reps[0]["cond"]) and reps[0]["cond"] >= 1.0
    expr = ("p_f * f_op_float32_madd + p_g * f_mem_access_global_float32 + p_s * f_mem_access_local_float32 + "
            "p_l * f_thread_groups")
    mm = pm.Model("f_wall_time", expr)
    Xm = np.array([mm.feature_values("mm_pf", n=n) for n in (256, 384, 512, 640, 768)])
    tm = np.array([1e-12 * n ** 3 + 3e-10 * n ** 2 for n in (256, 384, 512, 640, 768)])
    _, reps = pm.fit_batched([mm], [Xm], [tm])
    assert reps[0]["status"] == -5 and reps[0]["cond"] == float("inf")


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_ill_conditioned_linear_fit_matches_qr_oracle(eps):
    # two nearly collinear columns (condition number of the column-scaled
    # design ~1/eps): the library solves the normal equations in float-float
    # with iterative refinement, the oracle uses FP64 QR; they must agree
    dev()
    X = design(200, 91, nf=4)
    X[:, 3] = X[:, 2] * (1 + eps * pm_inputs.uniform((200,), 92, dtype=np.float64))
    expr = "p_a * f_sync_kernel_launch + p_b * f_thread_groups + p_c * f_op_float32_add + p_d * f_op_float32_mul"
    om = OModel("f_wall_time", expr)
    F = [dict(zip(om.features, r)) for r in X]
    ptrue = {"p_a": 5e-6, "p_b": 2e-9, "p_c": 3e-12, "p_d": 4e-12}
    t = np.array([om.eval(ptrue, f) for f in F]) * (1 + 1e-3 * pm_inputs.noise((200,), 93))
    m = pm.Model("f_wall_time", expr)
    assert m.features == om.features
    p, rep = m.fit(X, t)
    po, info = ofit.fit(om, F, t)
    assert rep["status"] == 0 and not info["rank_deficient"]
    A = X / t[:, None]
    An = A / np.linalg.norm(A, axis=0)
    kappa = np.linalg.cond(An)
    assert kappa > 0.1 / eps, kappa
    assert rep["cond"] <= kappa ** 2 * (1 + 1e-6)
    assert perr(p, po) <= 1e-6, (perr(p, po), kappa)


@pytest.mark.parametrize("p_edge,sigma,seed", [(1e5, 1e-2, 41), (1e7, 1e-2, 42), (1e5, 0.0, 43)])
def test_partial_overlap_model_default_start(p_edge, sigma, seed):
    # the suite's overlap-kernel model with the partial-overlap weight p_part
    # (a product of parameters, so its start-point column vanishes at the
    # origin and it starts from the clamp): features of the overlap kernel
    # for m = 0..32 local load-store pairs at two array sizes, outputs from
    # a generating point with 40 % of the smaller cost not hidden; the fit
    # from the default start must reach the oracle's optimum
    dev()
    from paper_1904_09538_gb300 import suite as S
    expr = S.overlap_model(partial=True)
    m = pm.Model("f_wall_time", expr)
    om = OModel("f_wall_time", expr)
    X = np.stack([oracle_row(om, "overlap", "N", N, 256, 1, 256, m=mm) for mm in range(33) for N in (2 ** 26, 2 ** 27)])
    truth = dict(p_launch=1.2e-5, p_gmem=1.2e-12, p_lmem=3e-12, p_edge=p_edge, p_part=0.4)
    t, om, F = synth(expr, X, truth, sigma, seed)
    assert m.features == om.features
    p, rep = m.fit(X, t)
    assert rep["status"] == 0 and rep["iterations"] < 200, rep
    po, _ = ofit.fit(om, F, t)
    pred = m.predict(p, X)
    pred_o = ofit.predict(om, po, F)
    assert np.max(np.abs(pred / pred_o - 1)) <= 1e-5
    i = m.params.index("p_part")
    assert abs(p[i] - po[om.params.index("p_part")]) <= 1e-3
    if sigma == 0.0:
        assert abs(p[i] - 0.4) <= 1e-3


def identified(om, F, t, po, eps_r=1e-13, bound=1e-7):
    """True when every parameter of the oracle's solution po is pinned well
    inside the 1e-6 bar by its own normal matrix: a perturbation of the
    relative residuals of eps_r per row (the float-float resolution both GPU
    paths compute at), aligned worst-case, moves parameter i by at most
    sqrt((A^-1)_ii) sqrt(l) eps_r in the scaled coordinates q = p / |po|
    (A = J^T J there); all of these must stay below `bound`."""
    _, J = ofit.residual_and_jacobian(om, F, t)
    Js = J(po) * np.abs(po)[None, :]
    Ainv = np.linalg.inv(Js.T @ Js)
    return bool(np.all(np.sqrt(np.diag(Ainv) * len(t)) * eps_r <= bound))


def _workload_oracle():
    from paper_1904_09538_gb300.fitbench import problem
    models, Xs, ts, p0s, ls = problem(64)
    refs = []
    for m, X, t, p0 in zip(models, Xs, ts, p0s):
        om = OModel("f_wall_time", m.expr)
        F = [dict(zip(om.features, row)) for row in X]
        po, _ = ofit.fit(om, F, t, p0=p0)
        refs.append((om, F, po, identified(om, F, t, po)))
    return models, Xs, ts, p0s, refs


def _grade_workload(models, Xs, ps, refs):
    """Worst parameter error over the identified models, worst prediction
    error over the others (none today: every model of the workload is
    identified)."""
    wp, wpred, unidentified = 0.0, 0.0, []
    for k, (m, X, p, (om, F, po, ok)) in enumerate(zip(models, Xs, ps, refs)):
        if ok:
            wp = max(wp, perr(p, po))
        else:
            unidentified.append(k)
            pred_o = np.asarray(ofit.predict(om, po, F))
            wpred = max(wpred, float(np.max(np.abs(m.predict(p, X) / pred_o - 1))))
    return wp, wpred, unidentified


def test_fit_workload_batched_matches_oracle():
    # the batched-fit workload the bench times: 64 models of 4..12
    # parameters (linear and tanh-overlap), 40..400 rows, one batched plan;
    # every fit converges to the oracle's parameters within 1e-6
    dev()
    models, Xs, ts, p0s, refs = _workload_oracle()
    assert {len(m.params) for m in models} == set(range(4, 13))
    ps, reps = pm.fit_batched(models, Xs, ts, p0s)
    assert all(r["status"] == 0 for r in reps), [r["status"] for r in reps]
    wp, wpred, unidentified = _grade_workload(models, Xs, ps, refs)
    assert unidentified == [], unidentified
    assert wp <= PTOL, wp


def test_fit_workload_plain_lm_matches_oracle():
    # the plain per-model fit the bench compares against, on the same 64
    # problems: host-driven LM through the autograd.Function, one model at
    # a time, at the same 1e-6 parameter bar
    d = dev()
    models, Xs, ts, p0s, refs = _workload_oracle()
    ps = []
    for m, X, t, p0 in zip(models, Xs, ts, p0s):
        p, rep = pag.lm_fit(m, torch.from_numpy(X).to(d), torch.from_numpy(t).to(d), p0)
        assert rep["status"] == 0, rep
        ps.append(p)
    wp, wpred, unidentified = _grade_workload(models, Xs, ps, refs)
    assert unidentified == [] and wp <= PTOL, (wp, unidentified)


def test_start_point_matches_oracle():
    # max_iter = 0 returns the library start point: the linear fit with every
    # tanh switch at 1/2, non-positive coefficients replaced by 1e-3 sum(t) /
    # sum |column| (1e-3 max |p| for a zero column), p_edge = 10 / median(t);
    # cases: no replacement, three replaced (the nine-parameter model), and a
    # column zero at the origin (p_part of the partial-overlap model)
    dev()
    from paper_1904_09538_gb300 import suite as S
    cases = []
    X = design(150, 9, nf=5)
    cases.append((OVL, X, synth(OVL, X, P_OVL, 1e-3, 10)[0]))
    X = design(300, 31, nf=8)
    cases.append((OVL_BIG, X, synth(OVL_BIG, X, P_BIG, 1e-2, 131)[0]))
    expr = S.overlap_model(partial=True)
    X = np.stack([oracle_row(OModel("f_wall_time", expr), "overlap", "N", N, 256, 1, 256, m=mm)
                  for mm in range(33) for N in (2 ** 26, 2 ** 27)])
    truth = dict(p_launch=1.2e-5, p_gmem=1.2e-12, p_lmem=3e-12, p_edge=1e5, p_part=0.4)
    cases.append((expr, X, synth(expr, X, truth, 1e-2, 41)[0]))
    replaced = []
    for expr, X, t in cases:
        m = pm.Model("f_wall_time", expr)
        om = OModel("f_wall_time", expr)
        F = [dict(zip(om.features, row)) for row in X]
        p, rep = m.fit(X, t, max_iter=0)
        assert rep["status"] == -4 and rep["iterations"] == 0
        po = ofit.start_point(om, F, t)
        assert perr(p, po) <= 1e-5, (expr[:40], perr(p, po), p, po)
        lin = OModel("f_wall_time", ofit._strip_tanh(expr))
        pl, _ = ofit.fit_linear(ofit.linear_design(lin, F), t)
        replaced.append(int(np.sum(pl <= 0)))
    assert replaced[0] == 0 and replaced[1] == 3 and replaced[2] >= 1
