"""Oracle: model calibration in FP64 (test infrastructure only).

Section "Computing Model Parameters": minimise || g(p) - t ||_2 over the
parameters, with the Jacobian j_ki = d g_k / d p_i from symbolic
differentiation, by Levenberg-Marquardt (SciPy's ``optimize.leastsq``, the
routine the paper names); ``scale_features_by_output()`` divides each row by
its output so the fit minimises relative error (used in all of the paper's
examples).

Readings of the paper taken here where it is silent or ambiguous:
  * relative residual r_k = 1 - g(p; f_k) / t_k with the features left
    unscaled inside g -- identical to dividing features by t_k for models
    linear in the features, and well defined for the tanh overlap model;
  * a model linear in its parameters is solved directly as a linear least
    squares problem on the column-scaled matrix X_ki / t_k (columns scaled to
    unit 2-norm); if its numerical rank (singular values above
    max(l, m) * eps * sigma_max) is below m the minimum-norm solution in the
    column-scaled coordinates is returned with rank_deficient = True;
  * the LM start point, when not given, is the linear fit of the model with
    every tanh switch replaced by 1/2, and p_edge0 = 10 / median(t); a
    coefficient that comes out non-positive is replaced by
    1e-3 * sum_k t_k / sum_k |h_ki| (h_i its column of that linear design),
    so that its term carries about 0.1 % of the outputs; for a column that
    is zero at the origin (a parameter that only multiplies others) the same
    rule uses its column at the point reached so far (1e-3 * max |p| if that
    is zero too);
  * LM iterates in scaled coordinates q = p / |p0| (the minimiser does not
    depend on the coordinates).

Geometric mean of relative error (Section "Results"):
    exp(mean(log(|t_hat - t| / t))).
"""
import math

import numpy as np
import scipy.optimize

from .model import Model


def linear_design(model, F):
    """For a model g = sum_i p_i * h_i(f) (linear in p), return H[l, m] with
    H[k, i] = h_i(f_k), obtained as dg/dp_i (exact for such models)."""
    l = len(F)
    H = np.zeros((l, len(model.params)))
    p0 = {name: 0.0 for name in model.params}
    for k in range(l):
        _, d = model.grad(p0, F[k])
        H[k] = d
    return H


def is_linear(model, F, probes=3, seed=7):
    """True when g is linear in p on these rows (checked at random points)."""
    rng = np.random.default_rng(seed)
    H = linear_design(model, F[:5])
    for _ in range(probes):
        p = {name: float(v) for name, v in zip(model.params, rng.standard_normal(len(model.params)))}
        for k in range(min(5, len(F))):
            g = model.eval(p, F[k])
            lin = float(np.dot(H[k], [p[n] for n in model.params]))
            if abs(g - lin) > 1e-9 * (abs(g) + sum(abs(H[k])) + 1e-300):
                return False
    return True


def fit_linear(H, t):
    """min_p sum_k (1 - H[k] . p / t_k)^2 via column-scaled least squares.

    Returns (p, info) with info = dict(rank, rank_deficient, residual, sv)."""
    H = np.asarray(H, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    A = H / t[:, None]
    cn = np.linalg.norm(A, axis=0)
    cn[cn == 0.0] = 1.0
    As = A / cn
    l, m = As.shape
    rcond = max(l, m) * np.finfo(np.float64).eps
    q, _, rank, sv = np.linalg.lstsq(As, np.ones(l), rcond=rcond)
    p = q / cn
    r = 1.0 - A @ p
    return p, dict(rank=int(rank), rank_deficient=bool(rank < m), residual=float(np.linalg.norm(r)),
                   sv=sv, colscale=cn)


def residual_and_jacobian(model, F, t):
    """Functions r(p_vec) and J(p_vec) for the relative residual
    r_k = 1 - g(p; f_k) / t_k (so J_ki = -dg_k/dp_i / t_k)."""
    names = model.params
    t = np.asarray(t, dtype=np.float64)

    def r(pv):
        p = dict(zip(names, pv))
        return np.array([1.0 - model.eval(p, F[k]) / t[k] for k in range(len(F))])

    def J(pv):
        p = dict(zip(names, pv))
        out = np.zeros((len(F), len(names)))
        for k in range(len(F)):
            _, d = model.grad(p, F[k])
            out[k] = -np.asarray(d) / t[k]
        return out
    return r, J


def start_point(model, F, t):
    """Start point: linear fit with every tanh(...) replaced by 0 (so each
    s_hat is 1/2); a non-positive coefficient becomes 1e-3 * sum(t) /
    sum |its column| (for a column zero at the origin, its column at the
    point reached so far; 1e-3 * max |p| if that is zero too); p_edge0 =
    10 / median(t)."""
    lin = Model(model.out_feature, _strip_tanh(model.expr))
    t = np.asarray(t, dtype=np.float64)
    p = {}
    if lin.params:
        H = linear_design(lin, F)
        pl, _ = fit_linear(H, t)
        big = max(1e-300, float(np.max(np.abs(pl))))
        tsum = float(np.sum(t))
        zero = []
        for i, (name, v) in enumerate(zip(lin.params, pl)):
            cs = float(np.sum(np.abs(H[:, i])))
            if v > 0:
                p[name] = v
            elif cs > 0:
                p[name] = 1e-3 * tsum / cs
            else:
                p[name] = 0.0
                zero.append(i)
        if zero:
            # a column that vanishes at the origin (a parameter that only
            # multiplies others): the same rule on its column at the point
            # reached so far (those parameters at 0)
            q = dict(p)
            cz = np.zeros(len(lin.params))
            for f in F:
                cz += np.abs(np.asarray(lin.grad(q, f)[1]))
            for i in zero:
                p[lin.params[i]] = 1e-3 * tsum / cz[i] if cz[i] > 0 else 1e-3 * big
    for name in model.params:
        if name not in p:
            p[name] = 10.0 / float(np.median(t))
    return np.array([p[n] for n in model.params])


def _strip_tanh(expr):
    out, i = [], 0
    while i < len(expr):
        if expr.startswith("tanh(", i):
            depth, j = 1, i + 5
            while depth:
                depth += {"(": 1, ")": -1}.get(expr[j], 0)
                j += 1
            out.append("0")
            i = j
        else:
            out.append(expr[i])
            i += 1
    return "".join(out)


def fit(model, F, t, p0=None, max_iter=200):
    """Calibrate `model` on rows F (list of {feature: value}) and outputs t.

    Linear-in-p models: direct least squares (fit_linear).  Otherwise
    Levenberg-Marquardt via scipy.optimize.leastsq with the analytic Jacobian.
    Returns (p_vec, info)."""
    t = np.asarray(t, dtype=np.float64)
    if is_linear(model, F):
        H = linear_design(model, F)
        p, info = fit_linear(H, t)
        info["method"] = "linear"
        return p, info
    r, J = residual_and_jacobian(model, F, t)
    if p0 is None:
        p0 = start_point(model, F, t)
    p0 = np.asarray(p0, dtype=np.float64)
    # solve in scaled coordinates q = p / |p0| (same minimiser; parameters
    # span many decades, e.g. 1e-12 s per operation next to p_edge ~ 1e4 / s)
    s = np.where(p0 != 0.0, np.abs(p0), 1.0)
    q, cov, infodict, mesg, ier = scipy.optimize.leastsq(
        lambda q: r(q * s), p0 / s, Dfun=lambda q: J(q * s) * s[None, :], full_output=True, ftol=1e-15,
        xtol=1e-15, gtol=0.0, maxfev=max_iter * (len(p0) + 1))
    p = q * s
    res = r(p)
    return p, dict(method="lm", ier=int(ier), nfev=int(infodict["nfev"]), residual=float(np.linalg.norm(res)),
                   message=mesg, rank_deficient=False)


def predict(model, p_vec, F):
    p = dict(zip(model.params, p_vec))
    return np.array([model.eval(p, f) for f in F])


def geomean_rel_err(pred, meas):
    pred = np.asarray(pred, dtype=np.float64)
    meas = np.asarray(meas, dtype=np.float64)
    e = np.abs(pred - meas) / meas
    return float(math.exp(np.mean(np.log(e))))


def geomean(values):
    """Geometric mean (the 'Mean' rows of the paper's accuracy tables)."""
    v = np.asarray(values, dtype=np.float64)
    return float(math.exp(np.mean(np.log(v))))


def fit_rows(job):
    """fit() of a model given by its expression on a feature matrix:
    job = (expression, feature names, rows (l x nf), t, p0).  A plain
    function of plain data, so that a process pool can run it.  Returns
    (p_vec, info)."""
    from .model import Model
    expr, names, rows, t, p0 = job
    m = Model("f_wall_time", expr)
    return fit(m, [dict(zip(names, r)) for r in rows], t, p0=p0)
