"""Oracle PDCS solver: Algorithm 2 wrapped around Algorithm 1 of the paper, step by
step, in plain FP64 (test infrastructure only; slow on purpose; recomputes
G x and G^T y from their definitions at every use).

Paper passages followed (section / equation / algorithm):
  * one PDHG step, eq. PDHG (Sec. 1.2);
  * AdaptiveStepPDHG, Function 1 and eq. adaptive_step_size (Sec. 2.1);
  * reflection parameter, eq. adaptive_reflection with maxErr, eq. tolerance (Sec. 2.2);
  * reflected Halpern step and weighted average, Algorithm 1 (Sec. 2);
  * normalized duality gap rho^N, Definition 2.1, and its bisection, Algorithm 3,
    eqs. compute_rho / compute_zt_2 (Sec. 2.4);
  * restart candidate and the three restart conditions, KKT_omega fallback (Sec. 2.3);
  * primal weight initialisation / update / reset (Sec. 2.5);
  * rescaling and unscaling, Algorithm 2 (Sec. 2.6);
  * termination, eq. PDCS_terminate_tolerance_rel (Sec. 3.2.3), exit codes Table 1.

Readings where the paper is silent or inconsistent:
  c3  kbar is incremented at the start of every attempt (accepted or rejected)
      before the step-size formula uses (kbar + 1).
  c4  eta_bar = +inf when (Delta y)^T G (Delta x) = 0.
  c5  the average is over the Halpern iterates z^{t,i}, weights eta^{t,i}.
  c6  method 'average' compares both candidates; 'halpern' always takes z.
  c7  restart / termination checks every check_freq accepted iterations (global
      count); beta needs maxErr(zhat) every iteration.
  c8  in the first restart period there is no reference gap: only condition 3.
  c9  bisection: t0 = r / sqrt(tau ||b1||^2 + sigma ||b2||^2) (the unconstrained
      step reaching radius r), at most 64 doublings, bisection until
      t_right - t_left <= bisect_rel_tol * t_right (default 1e-3; at most 64
      halvings); the value is returned at the last probe; r = 0 or b = 0
      give 0.
  c10 if any gap value used at a check is negative, every gap at that check is
      replaced by KKT_omega.
  c11 beta / maxErr / KKT_omega / rho^N use the rescaled problem; termination
      uses the unscaled problem with infinity norms.
  c15 the candidate is tested for termination and returned.
  ref the reference gap of a restart period is the candidate's gap at the check
      that started the period; N uses the last accepted step size.
  c19 infeasibility (Sec. 3.2.3 eps_*_infeasible_* options) is tested at every
      check after the optimality test, on the change of the restart candidate
      since the previous check (the direction in which the iterates of an
      infeasible problem diverge), with the paper's ratios taken on the
      homogeneous problem: err_abs,d (c = 0, plus the dual-cone violation of
      the y change) over the dual objective, and err_rel,p (h = 0, plus the
      violation of the recession cone of X by the x change) over -c^T x
      (kkt.infeasibility_ratios).  Taken on the candidate itself the ratio
      err_abs,d / (dual objective) is 0 for every y when all bounds are
      finite, so it would call feasible problems infeasible.  High accuracy:
      the ratio test alone (exit 3 / 5); low accuracy: also a rising trend,
      the candidates' dual objective (resp. -c^T x) strictly increasing over
      the last INFEAS_TREND_CHECKS checks (exit 2 / 4).
  c21 use_adaptive_step_size_weight = False: every attempt is accepted with
      the fixed step eta = 1 / sqrt(||G||_1 ||G||_inf) (induced norms: largest
      column / row absolute sum), an upper bound on 1 / ||G||_2, so that
      tau sigma ||G||_2^2 <= 1.
  c22 restart criteria: at multiples of check_freq (the duality-gap restart
      frequency) with use_duality_gap_restart the criterion is rho^N; at
      multiples of kkt_restart_freq with use_kkt_restart (and not a gap check)
      it is KKT_omega, as in the fallback of reading c10; at other checks
      (termination only) restart condition 3 alone can fire.  A gap that was
      not computed (a KKT-criterion check) counts like a negative one for c10.
"""
import time

import numpy as np

from .cones import proj_box, proj_cone_product
from .kkt import scaled_errors, unscaled_errors, kkt_omega, infeasibility_ratios
from .problem import ScaledProblem, apply_block_T

EXIT_OPTIMAL, EXIT_MAX_ITER, EXIT_TIME_LIMIT, EXIT_NUMERICAL = 0, 1, 6, 8
EXIT_PRIMAL_INFEAS_LOW, EXIT_PRIMAL_INFEAS_HIGH = 2, 3
EXIT_DUAL_INFEAS_LOW, EXIT_DUAL_INFEAS_HIGH = 4, 5
INFEAS_TREND_CHECKS = 3          # reading c19

# Restart thresholds of Sec. 2.3 and the primal-weight constants of Sec. 2.5.
BETA_SUFFICIENT, BETA_NECESSARY, BETA_ARTIFICIAL = 0.4, 0.8, 0.223
PW_THETA, PW_GUARD, PW_MAX, PW_MIN = 0.5, 1e-10, 1e5, 1e-5


# -- controller scalars (each is pinned by hand-derived values in the tests) --
def step_bound(dx2, dy2, inter, omega):
    """eta_bar of Function 1: (1/2) ||(dx, dy)||_omega^2 / |dy^T G dx| with
    ||z||_omega^2 = omega ||dx||^2 + ||dy||^2 / omega (eq. adaptive_step_size);
    +inf when the product vanishes (reading c4)."""
    inter = abs(inter)
    num = 0.5 * (omega * dx2 + dy2 / omega)
    return num / inter if inter > 0 else np.inf


def next_step_size(eta, eta_bar, kbar):
    """eta' of Function 1; kbar already counts the current attempt (reading c3)."""
    return min((1.0 - (kbar + 1) ** -0.3) * eta_bar, (1.0 + (kbar + 1) ** -0.6) * eta)


def reflection(max_err):
    """Reflection parameter, eq. adaptive_reflection: Proj_[0,1](-0.1 log10(maxErr) + 0.2)."""
    if max_err <= 0:
        return 1.0
    return float(min(1.0, max(0.0, -0.1 * np.log10(max_err) + 0.2)))


def halpern_step(k, beta, zhat, z, z0):
    """Reflected Halpern step of Algorithm 1:
    (k+1)/(k+2) ((1+beta) zhat - beta z) + z0 / (k+2)."""
    a = (k + 1.0) / (k + 2.0)
    return a * ((1.0 + beta) * zhat - beta * z) + z0 / (k + 2.0)


def initialize_primal_weight(c_norm, h_norm):
    """InitializePrimalWeight of Sec. 2.5 from ||c||_2 and ||h||_2."""
    return c_norm / h_norm if (c_norm > PW_GUARD and h_norm > PW_GUARD) else 1.0


def primal_weight_update(dx, dy, omega, omega0):
    """PrimalWeightUpdate of Sec. 2.5 (theta = 0.5) with the reset to omega0
    outside [1e-5, 1e5]; dx, dy = ||x^{t,0} - x^{t-1,0}||, ||y^{t,0} - y^{t-1,0}||."""
    if dx > PW_GUARD and dy > PW_GUARD:
        omega = float(np.exp(PW_THETA * np.log(dy / dx) + (1.0 - PW_THETA) * np.log(omega)))
    if omega > PW_MAX or omega < PW_MIN:
        omega = omega0
    return omega


def restart_conditions(val, ref, prev, k, kbar):
    """The three restart conditions of Sec. 2.3 for the candidate's measure val
    against the anchor's ref (None in the first period, reading c8) and the
    previous candidate's prev (None if none yet in this period); k = inner
    iterations, kbar = all attempts.  Returns (sufficient, necessary, long)."""
    cond3 = k >= BETA_ARTIFICIAL * kbar
    if ref is None:
        return False, False, cond3
    cond1 = val <= BETA_SUFFICIENT * ref
    cond2 = (prev is not None) and val <= BETA_NECESSARY * ref and val > prev
    return cond1, cond2, cond3


def fixed_step_size(G):
    """Step of the non-adaptive mode (reading c21): 1 / sqrt(||G||_1 ||G||_inf)."""
    if G.nnz == 0:
        return 1.0
    A = abs(G)
    n1 = float(np.max(np.asarray(A.sum(axis=0)).ravel()))
    ninf = float(np.max(np.asarray(A.sum(axis=1)).ravel()))
    return 1.0 / np.sqrt(n1 * ninf)


def _rising(seq, count):
    s = seq[-(count + 1):]
    return len(s) == count + 1 and all(b > a for a, b in zip(s, s[1:]))


def infeasibility_exit(ratios, dobj_hist, mpobj_hist, opts):
    """Sec. 3.2.3 infeasibility tests (reading c19): ratios = (primal, dual)
    ratio of the candidate's change since the previous check
    (kkt.infeasibility_ratios); dobj_hist / mpobj_hist hold the dual
    objective / -c^T x of the candidates of every check so far, this one
    included.  Returns an exit code of Table 1 (2 to 5) or None."""
    pr, dr = ratios
    if pr < opts.eps_primal_infeasible_high_acc:
        return EXIT_PRIMAL_INFEAS_HIGH
    if dr < opts.eps_dual_infeasible_high_acc:
        return EXIT_DUAL_INFEAS_HIGH
    if pr < opts.eps_primal_infeasible_low_acc and _rising(dobj_hist, INFEAS_TREND_CHECKS):
        return EXIT_PRIMAL_INFEAS_LOW
    if dr < opts.eps_dual_infeasible_low_acc and _rising(mpobj_hist, INFEAS_TREND_CHECKS):
        return EXIT_DUAL_INFEAS_LOW
    return None


class Options:
    """Solver options; names follow the paper's direct API (Sec. 3.2.3)."""

    def __init__(self, **kw):
        self.rel_tol = 1e-6
        self.abs_tol = 1e-6
        self.require_abs = False
        self.time_limit = 1000.0
        self.max_iter = 1 << 62
        self.use_preconditioner = True
        self.ruiz_iters = 10
        self.pc_alpha = 1.0
        self.method = "average"
        self.use_adaptive_restart = True
        self.check_freq = 64                 # duality-gap restart / termination period
        self.bisect_rel_tol = 1e-3          # reading c9
        self.use_adaptive_step_size_weight = True
        self.use_duality_gap_restart = True
        self.use_kkt_restart = False
        self.kkt_restart_freq = 2000
        self.eps_primal_infeasible_low_acc = 1e-12
        self.eps_dual_infeasible_low_acc = 1e-12
        self.eps_primal_infeasible_high_acc = 1e-16
        self.eps_dual_infeasible_high_acc = 1e-16
        for k, v in kw.items():
            if not hasattr(self, k):
                raise KeyError(k)
            setattr(self, k, v)


class Oracle:
    """State and steps of Algorithm 1 on a ScaledProblem."""

    def __init__(self, prob, opts=None):
        self.opts = opts or Options()
        o = self.opts
        self.sp = ScaledProblem(prob, o.use_preconditioner, o.ruiz_iters, o.pc_alpha)
        sp_ = self.sp
        # Sec. 2.5 InitializePrimalWeight on the rescaled data.
        self.omega0 = initialize_primal_weight(np.linalg.norm(sp_.c), np.linalg.norm(sp_.h))
        # Algorithm 1 Require: eta_hat = 1 / ||G||_inf (reading c2: max |entry|).
        gmax = np.max(np.abs(sp_.G.data)) if sp_.G.nnz else 1.0
        self.eta0 = 1.0 / gmax
        self.eta_fixed = fixed_step_size(sp_.G)                    # reading c21

    # -- projections onto X = [lhat, uhat] x D2^{-1} K_p and Y = (D1 K_r)^* ----
    def proj_X(self, v):
        sp_ = self.sp
        out = np.empty_like(v)
        out[:sp_.nb] = proj_box(v[:sp_.nb], sp_.lo, sp_.hi)
        out[sp_.nb:] = proj_cone_product(v[sp_.nb:], sp_.col_cones, 1.0 / sp_.d2[sp_.nb:])
        return out

    def proj_Y(self, v):
        sp_ = self.sp
        return proj_cone_product(v, sp_.row_cones, 1.0 / sp_.d1, dual=True)

    # -- eq. PDHG ---------------------------------------------------------------
    def one_pdhg(self, x, y, tau, sigma):
        sp_ = self.sp
        xh = self.proj_X(x - tau * (sp_.c - sp_.GT @ y))
        yh = self.proj_Y(y + sigma * (sp_.h - sp_.G @ (2.0 * xh - x)))
        return xh, yh

    # -- Function 1 ----------------------------------------------------------
    def adaptive_step(self, x, y, omega, eta, kbar):
        sp_ = self.sp
        if not self.opts.use_adaptive_step_size_weight:              # reading c21
            kbar += 1
            eta = self.eta_fixed
            xh, yh = self.one_pdhg(x, y, eta / omega, eta * omega)
            return xh, yh, eta, eta, kbar
        while True:
            kbar += 1                                                # reading c3
            xh, yh = self.one_pdhg(x, y, eta / omega, eta * omega)
            dx = xh - x
            dy = yh - y
            eta_bar = step_bound(float(dx @ dx), float(dy @ dy), float(dy @ (sp_.G @ dx)), omega)
            eta_p = next_step_size(eta, eta_bar, kbar)
            if eta < eta_bar:
                return xh, yh, eta, eta_p, kbar
            eta = eta_p

    # -- eq. adaptive_reflection ----------------------------------------------
    @staticmethod
    def reflection(max_err):
        return reflection(max_err)

    # -- Definition 2.1 / Algorithm 3 ------------------------------------------
    def normalized_gap(self, x, y, r, tau, sigma):
        sp_ = self.sp
        if r <= 0:
            return 0.0
        b1 = sp_.GT @ y - sp_.c
        b2 = sp_.h - sp_.G @ x
        scale = np.sqrt(tau * float(b1 @ b1) + sigma * float(b2 @ b2))
        if scale <= 0:
            return 0.0

        def z_of(t):
            return self.proj_X(x + t * tau * b1), self.proj_Y(y + t * sigma * b2)

        def dist(xt, yt):
            return np.sqrt(float((xt - x) @ (xt - x)) / tau + float((yt - y) @ (yt - y)) / sigma)

        t = r / scale
        t_left, t_right = 0.0, t
        for k in range(64):
            xt, yt = z_of(t)
            if dist(xt, yt) > r:
                if k == 0:
                    t_left, t_right = 0.0, t
                else:
                    t_left, t_right = 0.5 * t, t
                break
            t = 2.0 * t
            t_left, t_right = 0.5 * t, t
        for _ in range(64):
            if t_right - t_left <= self.opts.bisect_rel_tol * t_right:
                break
            t_mid = 0.5 * (t_left + t_right)
            xt, yt = z_of(t_mid)
            if dist(xt, yt) < r:
                t_left = t_mid
            else:
                t_right = t_mid
        return (float(b1 @ (xt - x)) + float(b2 @ (yt - y))) / r

    @staticmethod
    def n_norm(dx, dy, tau, sigma):
        return float(np.sqrt(float(dx @ dx) / tau + float(dy @ dy) / sigma))

    # -- Algorithm 1 / 2 --------------------------------------------------------
    def solve(self, x0=None, y0=None, trace=None, snapshots=None, states=None, init_state=None):
        """Run the solver.  trace: list to append one dict per accepted iteration.
        snapshots: dict {iteration: None} filled with copies of the scaled
        Halpern iterate (x, y) after that many accepted iterations.
        states: dict {iteration: None} filled with the complete solver state
        after that many accepted iterations (0 = before the first one).
        init_state: a state in the form `states` records, to continue from
        (the infeasibility history starts empty)."""
        o = self.opts
        sp_ = self.sp
        t_start = time.perf_counter()
        # Warm start given in the original variables: undo the RSOC rotation
        # (an involution) and the rescaling (Algorithm 2).
        x = np.zeros(sp_.n) if x0 is None else apply_block_T(np.asarray(x0, float), sp_.col_T) / sp_.d2
        y = np.zeros(sp_.m) if y0 is None else apply_block_T(np.asarray(y0, float), sp_.row_T) / sp_.d1
        xa, ya = x.copy(), y.copy()            # anchor z^{t,0}
        omega = self.omega0
        eta_hat = self.eta0 if o.use_adaptive_step_size_weight else self.eta_fixed
        kbar = 0
        it = 0                                  # accepted iterations, all periods
        t_period = 0
        k = 0
        wsum = 0.0
        xs = np.zeros(sp_.n)
        ys = np.zeros(sp_.m)
        rho_ref = None                          # (rho, errs) of the anchor
        prev = None                             # (rho, errs) of previous candidate
        restarts = 0
        xc, yc = x.copy(), y.copy()
        exit_code = None
        eta = eta_hat
        dobj_hist, mpobj_hist = [], []          # candidates' objectives (reading c19)
        any_check = False
        last_cand = None                        # candidate of the previous check

        def capture():
            return dict(x=x.copy(), y=y.copy(), x0=xa.copy(), y0=ya.copy(), xs=xs.copy(),
                        ys=ys.copy(), wsum=wsum, k=k, kbar=kbar, iter=it, period=t_period,
                        restarts=restarts, eta_hat=eta_hat, eta=eta, omega=omega,
                        has_ref=rho_ref is not None,
                        ref=(rho_ref[0], rho_ref[1]["abs_p"], rho_ref[1]["abs_d"],
                             rho_ref[1]["abs_gap"]) if rho_ref is not None else (0.0,) * 4,
                        has_prev=prev is not None,
                        prev=(prev[0], prev[1]["abs_p"], prev[1]["abs_d"], prev[1]["abs_gap"])
                        if prev is not None else (0.0,) * 4)

        if init_state is not None:
            st = init_state
            x, y = st["x"].copy(), st["y"].copy()
            xa, ya = st["x0"].copy(), st["y0"].copy()
            xs, ys = st["xs"].copy(), st["ys"].copy()
            wsum, k, kbar, it = st["wsum"], st["k"], st["kbar"], st["iter"]
            t_period, restarts = st["period"], st["restarts"]
            eta_hat, eta, omega = st["eta_hat"], st["eta"], st["omega"]
            errs = lambda t: dict(abs_p=t[1], abs_d=t[2], abs_gap=t[3])  # noqa: E731
            rho_ref = (st["ref"][0], errs(st["ref"])) if st["has_ref"] else None
            prev = (st["prev"][0], errs(st["prev"])) if st["has_prev"] else None
            xc, yc = x.copy(), y.copy()
        if states is not None and 0 in states:
            states[0] = capture()
        while True:
            xh, yh, eta, eta_hat, kbar = self.adaptive_step(x, y, omega, eta_hat, kbar)
            errh = scaled_errors(sp_, xh, yh)
            beta = reflection(errh["max_err"])
            x = halpern_step(k, beta, xh, x, xa)
            y = halpern_step(k, beta, yh, y, ya)
            wsum += eta
            xs += eta * x
            ys += eta * y
            k += 1
            it += 1
            rec = dict(iter=it, kbar=kbar, period=t_period, eta=eta, eta_hat=eta_hat, beta=beta,
                       omega=omega, max_err=errh["max_err"], check=0, cand_avg=-1,
                       restart=0, rho_c=np.nan, fallback=0)
            gap_check = o.use_duality_gap_restart and it % o.check_freq == 0
            kkt_check = o.use_kkt_restart and it % o.kkt_restart_freq == 0
            if it % o.check_freq == 0 or kkt_check:
                rec["check"] = 1
                any_check = True
                tau, sigma = eta / omega, eta * omega
                xbar, ybar = xs / wsum, ys / wsum
                avg = o.method == "average"
                err_h = scaled_errors(sp_, x, y)
                err_a = scaled_errors(sp_, xbar, ybar) if avg else None
                if gap_check:
                    r_h = self.n_norm(x - xa, y - ya, tau, sigma)
                    rho_h = self.normalized_gap(x, y, r_h, tau, sigma)
                    if avg:
                        r_a = self.n_norm(xbar - xa, ybar - ya, tau, sigma)
                        rho_a = self.normalized_gap(xbar, ybar, r_a, tau, sigma)
                    else:
                        rho_a = np.inf
                else:
                    rho_h = np.nan                                   # reading c22
                    rho_a = np.nan if avg else np.inf
                used = [rho_h] + ([rho_a] if avg else [])
                if rho_ref is not None:
                    used.append(rho_ref[0])
                if prev is not None:
                    used.append(prev[0])
                fallback = any(not (v >= 0) for v in used)           # readings c10, c22
                rec["fallback"] = int(fallback)
                if fallback:
                    m_h = kkt_omega(err_h, omega)
                    m_a = kkt_omega(err_a, omega) if err_a is not None else np.inf
                else:
                    m_h, m_a = rho_h, rho_a
                if m_h <= m_a:
                    xc, yc, rho_c, err_c, cand_avg = x.copy(), y.copy(), rho_h, err_h, 0
                    val_c = m_h
                else:
                    xc, yc, rho_c, err_c, cand_avg = xbar, ybar, rho_a, err_a, 1
                    val_c = m_a
                rec["cand_avg"] = cand_avg
                rec["rho_c"] = val_c
                ue = unscaled_errors(sp_, xc, yc)
                done = ue["max_rel"] <= o.rel_tol and (not o.require_abs or max(
                    ue["abs_p"], ue["abs_d"], ue["abs_gap"]) <= o.abs_tol)
                dobj_hist.append(ue["dobj"])
                mpobj_hist.append(-ue["pobj"])
                if done:
                    exit_code = EXIT_OPTIMAL
                elif not np.isfinite(ue["max_rel"]):
                    exit_code = EXIT_NUMERICAL
                elif last_cand is not None:
                    ratios = infeasibility_ratios(sp_, xc - last_cand[0], yc - last_cand[1])
                    rec["infeas"] = ratios
                    exit_code = infeasibility_exit(ratios, dobj_hist, mpobj_hist, o)
                last_cand = (xc.copy(), yc.copy())
                if exit_code is None:
                    do_restart = False
                    if o.use_adaptive_restart:
                        ref = pv = None                               # reading c8
                        if rho_ref is not None:
                            ref = kkt_omega(rho_ref[1], omega) if fallback else rho_ref[0]
                        if prev is not None:
                            pv = kkt_omega(prev[1], omega) if fallback else prev[0]
                        cond1, cond2, cond3 = restart_conditions(val_c, ref, pv, k, kbar)
                        if not (gap_check or kkt_check):
                            cond1 = cond2 = False                     # reading c22
                        do_restart = cond1 or cond2 or cond3
                    if do_restart:
                        rec["restart"] = 1
                        dx = np.linalg.norm(xc - xa)
                        dy = np.linalg.norm(yc - ya)
                        omega = primal_weight_update(dx, dy, omega, self.omega0)
                        rho_ref = (rho_c, err_c)
                        prev = None
                        xa, ya = xc.copy(), yc.copy()
                        x, y = xc.copy(), yc.copy()
                        k = 0
                        wsum = 0.0
                        xs[:] = 0.0
                        ys[:] = 0.0
                        t_period += 1
                        restarts += 1
                    else:
                        prev = (rho_c, err_c)
            if trace is not None:
                trace.append(rec)
            if snapshots is not None and it in snapshots:
                snapshots[it] = (x.copy(), y.copy())
            if states is not None and it in states:
                states[it] = capture()
            if exit_code is not None:
                break
            if it >= o.max_iter:
                exit_code = EXIT_MAX_ITER
                break
            if time.perf_counter() - t_start > o.time_limit:
                exit_code = EXIT_TIME_LIMIT
                break
        if exit_code not in (EXIT_OPTIMAL, EXIT_PRIMAL_INFEAS_LOW, EXIT_PRIMAL_INFEAS_HIGH,
                             EXIT_DUAL_INFEAS_LOW, EXIT_DUAL_INFEAS_HIGH):
            # Return the most recent candidate; before the first check, z itself.
            if not any_check:
                xc, yc = x.copy(), y.copy()
        ue = unscaled_errors(sp_, xc, yc)
        xo = apply_block_T(ue["x"], sp_.col_T)
        yo = apply_block_T(ue["y"], sp_.row_T)
        prob = sp_.orig
        s = prob.G @ xo - prob.h
        return dict(exit_code=exit_code, x=xo, y=yo, s=s, pobj=ue["pobj"], dobj=ue["dobj"],
                    err_rel_p=ue["rel_p"], err_rel_d=ue["rel_d"], err_rel_gap=ue["rel_gap"],
                    err_abs_p=ue["abs_p"], err_abs_d=ue["abs_d"], err_abs_gap=ue["abs_gap"],
                    iters=it, attempts=kbar, restarts=restarts,
                    solve_time_s=time.perf_counter() - t_start,
                    x_scaled=x, y_scaled=y, omega=omega, eta_hat=eta_hat)


def solve(prob, x0=None, y0=None, trace=None, snapshots=None, states=None, init_state=None,
          **opts):
    """Convenience wrapper: Oracle(prob, Options(**opts)).solve(...)."""
    return Oracle(prob, Options(**opts)).solve(x0, y0, trace, snapshots, states, init_state)
