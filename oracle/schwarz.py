"""Two-level nonlinear Schwarz (one-level, additive, hybrid) in plain FP64 (oracle, CPU).

Test infrastructure: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg.

The method follows Section 2 of the paper:

* local corrections T_i(u): the solution of R_i F(u - P_i T_i(u)) = 0 (Eq. 4), computed by a
  local Newton loop in the variable w = R_i u - T_i (so T_i = R_i u - w);
* F_1(u) = sum_i P~_i T_i(u) (Eq. 5 with the restricted extension of Eq. 8, RASPEN);
* coarse correction T_0(u): R_0 F(u - P_0 T_0(u)) = 0 with R_0 = P_0^T (Eq. 9), Newton in c;
* F_a(u) = sum_i P~_i T_i(u) + P_0 T_0(u) (Eq. 10), F_h(u) = sum_i P~_i T_i(u_0) + P_0 T_0(u),
  u_0 = u - P_0 T_0(u) (Eq. 11);
* exact tangents (Eqs. 6, 7, 12): Q_i(x) = P_i (R_i DF(x) P_i)^-1 R_i DF(x) with P~_i on the
  outside of every local term;
* the outer loop is Newton's method on F_x(u) = 0 with the tangent system of Eq. 13 solved
  by restarted GMRES, u <- u - du (optionally with backtracking on ||F_x||, a reading: the
  paper states no globalisation of the outer step);
* the coarse basis is built once from DF(u^(0)), or (option, a reading) rebuilt from DF(u) at
  every outer iterate u;
* the stopping test of the outer loop uses the original residual, ||F(u)||_2 < tol.

Readings where the paper is silent: local and coarse
Newton stop at ||r|| <= max(1e-11, 1e-5 ||r_0||) (Section 3 tolerances), at most 50
iterations, Armijo backtracking with halving (at most 10 trial steps, sufficient decrease
1e-4 alpha); GMRES(50) with modified Gram-Schmidt and Givens rotations, zero initial guess,
relative tolerance 1e-6, at most 1000 iterations (Section 3); the coarse basis is built
once from DF(u^(0)).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2410_24138_gb300.inputs import Problem

from . import coarse as coarse_mod
from . import decomposition as dec
from . import fem

ONE_LEVEL, ADDITIVE, HYBRID = "one", "add", "hybrid"

STATUS_CONVERGED = 0
STATUS_MAXIT = 1
STATUS_LINESEARCH = 2
STATUS_NONFINITE = 3


@dataclasses.dataclass
class Options:
    coupling: str = HYBRID
    inner_rtol: float = 1e-5
    inner_atol: float = 1e-11
    inner_maxit: int = 50
    ls_trials: int = 10
    armijo: float = 1e-4
    gmres_rtol: float = 1e-6
    gmres_restart: int = 50
    gmres_maxit: int = 1000
    outer_atol: float = 1e-8
    outer_maxit: int = 30
    load_steps: int = 1
    outer_backtrack: bool = False
    coarse_rebuild: bool = False


# ----------------------------------------------------------------------------------------------
# one Newton iteration rule, shared by the local, the coarse and the plain global solves
# ----------------------------------------------------------------------------------------------

def newton(x0, residual, solve_jacobian, opts: Options):
    """Damped Newton on r(x) = 0: x <- x - alpha * DF^-1 r.

    ``residual(x)`` returns (r, ok); ``solve_jacobian(x, r)`` returns DF(x)^-1 r.
    Stops when ||r|| <= max(atol, rtol ||r_0||).  Armijo backtracking: the first of
    alpha = 1, 1/2, ... (``ls_trials`` values) with finite r and
    ||r(x - alpha s)|| <= (1 - 1e-4 alpha) ||r(x)|| is taken.
    Returns (x, iterations, status, ||r_0||, ||r||).
    """
    x = x0.copy()
    r, ok = residual(x)
    rn = float(np.linalg.norm(r)) if ok else np.inf
    r0 = rn
    if not np.isfinite(rn):
        return x, 0, STATUS_NONFINITE, r0, rn
    tol = max(opts.inner_atol, opts.inner_rtol * r0)
    its = 0
    while rn > tol:
        if its >= opts.inner_maxit:
            return x, its, STATUS_MAXIT, r0, rn
        s = solve_jacobian(x, r)
        alpha = 1.0
        accepted = False
        for _ in range(opts.ls_trials):
            xt = x - alpha * s
            rt, ok = residual(xt)
            rtn = float(np.linalg.norm(rt)) if ok else np.inf
            if np.isfinite(rtn) and rtn <= (1.0 - opts.armijo * alpha) * rn:
                accepted = True
                break
            alpha *= 0.5
        its += 1
        if not accepted:
            return x, its, STATUS_LINESEARCH, r0, rn
        x, r, rn = xt, rt, rtn
    return x, its, STATUS_CONVERGED, r0, rn


# ----------------------------------------------------------------------------------------------
# local problems (Eq. 4)
# ----------------------------------------------------------------------------------------------

class LocalProblem:
    """R_i F(.) and R_i DF(.) of one overlapping subdomain, on its table of touched dofs."""

    def __init__(self, model: fem.Model, sub: dec.Subdomain):
        prob = model.prob
        self.model = model
        self.sub = sub
        nd = model.ndof
        self.Xe = prob.xy[sub.tnodes][sub.lconn]
        self.ldofs = (sub.lconn[:, :, None] * nd + np.arange(nd)[None, None, :]).reshape(sub.lconn.shape[0], -1)
        self.tdofs = sub.table_dofs(nd)
        self.nt = self.tdofs.shape[0]
        if sub.tedges.size:
            self.edofs = (sub.ledges[:, :, None] * nd + np.arange(nd)[None, None, :]).reshape(sub.ledges.shape[0], -1)
            self.Xedge = prob.xy[sub.tnodes][sub.ledges]
        else:
            self.edofs = None

    def table(self, u: np.ndarray, w: np.ndarray) -> np.ndarray:
        """Values on the table dofs: u outside V_i, w on V_i (the state u - P_i T_i)."""
        xt = u[self.tdofs].copy()
        xt[self.sub.tpos] = w
        return xt

    def residual(self, xt: np.ndarray, load: float):
        r, _, ok = self.model.element_terms(self.sub.elems, self.Xe, xt[self.ldofs], want_jac=False, load=load)
        full = np.zeros(self.nt)
        np.add.at(full, self.ldofs.ravel(), r.ravel())
        if self.edofs is not None:
            fe = self.model.external_load(self.sub.tedges, self.Xedge, load)
            np.add.at(full, self.edofs.ravel(), -fe.ravel())
        return full[self.sub.tpos], ok

    def jacobian_rows(self, xt: np.ndarray) -> sp.csr_matrix:
        """R_i DF(x): rows = local unknowns, columns = table dofs."""
        _, K, _ = self.model.element_terms(self.sub.elems, self.Xe, xt[self.ldofs], want_jac=True)
        nd = self.ldofs.shape[1]
        rows = np.repeat(self.ldofs, nd, axis=1).ravel()
        cols = np.tile(self.ldofs, (1, nd)).ravel()
        full = sp.coo_matrix((K.ravel(), (rows, cols)), shape=(self.nt, self.nt)).tocsr()
        return full[self.sub.tpos]

    def solve_newton(self, u: np.ndarray, w0: np.ndarray, opts: Options, load: float):
        """Local Newton for Eq. 4 started from w0.  Returns (w, its, status, r0, r)."""
        def residual(w):
            return self.residual(self.table(u, w), load)

        def solve_jac(w, r):
            J = self.jacobian_rows(self.table(u, w))[:, self.sub.tpos].tocsc()
            return spla.splu(J).solve(r)

        return newton(w0, residual, solve_jac, opts)


# ----------------------------------------------------------------------------------------------
# the solver state shared by F_x and its tangent
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class LocalResult:
    w: np.ndarray              # converged local state (v_i or u_i on V_i)
    T: np.ndarray              # T_i = R_i x - w, x the point the correction was taken at
    its: int
    status: int


class Schwarz:
    """Everything set up once per problem: model, subdomains, owners, coarse space."""

    def __init__(self, prob: Problem, opts: Options, with_coarse: bool | None = None, which=None):
        self.prob = prob
        self.opts = opts
        self.model = fem.Model(prob)
        self.N = prob.n_nodes * prob.ndof
        self.free = fem.free_mask(prob)
        self.subs, self.owner = dec.decompose(prob, which)
        self.locals = [LocalProblem(self.model, s) for s in self.subs]
        need_coarse = opts.coupling != ONE_LEVEL if with_coarse is None else with_coarse
        self.cs = None
        self.star = None
        if need_coarse:
            self.star = dec.node_star(prob.conn, prob.n_nodes)
            K0 = fem.global_jacobian(self.model, np.zeros(self.N))
            self.cs = coarse_mod.rgdsw_coarse_space(prob, self.star, K0)
        self.stats = {"subdomain_newton_steps": 0}

    # -- global residual and tangent --------------------------------------------------------
    def F(self, u, load=1.0):
        return fem.global_residual(self.model, u, load)

    def DF(self, u):
        return fem.global_jacobian(self.model, u)

    # -- local corrections ------------------------------------------------------------------
    def local_corrections(self, x: np.ndarray, load: float, guesses=None):
        out = []
        for i, lp in enumerate(self.locals):
            rx = x[lp.sub.dofs]
            w0 = rx if guesses is None or guesses[i] is None else guesses[i]
            w, its, status, _, _ = lp.solve_newton(x, w0, self.opts, load)
            self.stats["subdomain_newton_steps"] += its
            out.append(LocalResult(w, rx - w, its, status))
        return out

    def combine(self, results) -> np.ndarray:
        """sum_i P~_i T_i (injective: every free dof is written by its owner only)."""
        y = np.zeros(self.N)
        for lp, res in zip(self.locals, results):
            sub = lp.sub
            y[sub.dofs[sub.owned]] = res.T[sub.owned]
        return y

    # -- coarse correction (Eq. 9) ------------------------------------------------------------
    def coarse_correction(self, u: np.ndarray, load: float):
        P0 = self.cs.P0
        P0T = P0.T.tocsr()

        def residual(c):
            x = u - P0 @ c
            with np.errstate(invalid="ignore", divide="ignore"):
                F = self.F(x, load)
            return P0T @ F, bool(np.all(np.isfinite(F)))

        def solve_jac(c, g):
            # d/dc P0^T F(u - P0 c) = -P0^T DF P0 = -A0, so the Newton step is c <- c + A0^-1 g
            A0 = (P0T @ self.DF(u - P0 @ c) @ P0).toarray()
            return -np.linalg.solve(A0, g)

        c, its, status, _, _ = newton(np.zeros(P0.shape[1]), residual, solve_jac, self.opts)
        return c, its, status

    # -- F_x and everything its tangent needs -------------------------------------------------
    def evaluate(self, u: np.ndarray, load: float = 1.0, guesses=None):
        """F_x(u) for the configured coupling, plus the linearisation data of Eq. 12."""
        coupling = self.opts.coupling
        st = {"coupling": coupling, "u": u}
        if coupling == ONE_LEVEL:
            res = self.local_corrections(u, load, guesses)
            Fx = self.combine(res)
            points = u
        else:
            c, cits, cstatus = self.coarse_correction(u, load)
            P0c = self.cs.P0 @ c
            u0 = u - P0c
            st.update(c=c, coarse_its=cits, coarse_status=cstatus, u0=u0)
            points = u if coupling == ADDITIVE else u0
            res = self.local_corrections(points, load, guesses)
            Fx = self.combine(res) + P0c
        st["local"] = res
        st["Fx"] = Fx
        st["points"] = points
        return Fx, st

    def tangent(self, st):
        """Return v -> DF_x(u) v (Eq. 6 / Eq. 12) with P~_i outside the local terms."""
        locs = []
        for lp, res in zip(self.locals, st["local"]):
            xt = lp.table(st["points"], res.w)
            Jrows = lp.jacobian_rows(xt)
            lu = spla.splu(Jrows[:, lp.sub.tpos].tocsc())
            locs.append((lp, Jrows, lu))
        coupling = st["coupling"]
        coarse_apply = None
        if coupling != ONE_LEVEL:
            P0 = self.cs.P0
            J0 = self.DF(st["u0"])
            A0 = (P0.T @ J0 @ P0).toarray()

            def coarse_apply(v):
                return P0 @ np.linalg.solve(A0, P0.T @ (J0 @ v))

        def local_sum(v):
            y = np.zeros(self.N)
            for lp, Jrows, lu in locs:
                z = lu.solve(Jrows @ v[lp.tdofs])
                sub = lp.sub
                y[sub.dofs[sub.owned]] = z[sub.owned]
            return y

        def apply(v):
            v = np.where(self.free, v, 0.0)
            if coupling == ONE_LEVEL:
                return local_sum(v)
            w0 = coarse_apply(v)
            if coupling == ADDITIVE:
                return local_sum(v) + w0
            return local_sum(v - w0) + w0

        return apply

    # -- the outer Newton loop (Eq. 13) ---------------------------------------------------------
    def solve(self, u0: np.ndarray | None = None, log=None):
        opts = self.opts
        u = np.zeros(self.N) if u0 is None else u0.copy()
        history = []
        t0 = time.perf_counter()
        steps = max(1, opts.load_steps)
        for step in range(steps):
            load = (step + 1) / steps
            cached = None  # F_x and its linearisation at u, from the previous step's backtracking
            for k in range(opts.outer_maxit + 1):
                nF = float(np.linalg.norm(self.F(u, load)))
                if nF < opts.outer_atol or k == opts.outer_maxit:
                    break
                if cached is None and opts.coarse_rebuild and self.cs is not None:
                    # the coarse basis from the tangent at the current iterate (same interface values)
                    self.cs = coarse_mod.rgdsw_coarse_space(self.prob, self.star, self.DF(u))
                Fx, st = cached if cached is not None else self.evaluate(u, load)
                cached = None
                if not np.any(Fx):
                    break  # every correction is exactly zero: the iteration cannot move any more
                A = self.tangent(st)
                du, gits, gres = gmres(A, Fx, opts.gmres_rtol, opts.gmres_restart, opts.gmres_maxit)
                rec = {"load": load, "outer": k, "normF": nF, "normFx": float(np.linalg.norm(Fx)),
                       "gmres_its": gits, "gmres_relres": gres,
                       "local_its": [r.its for r in st["local"]],
                       "local_status": [r.status for r in st["local"]],
                       "coarse_its": st.get("coarse_its", 0), "coarse_status": st.get("coarse_status", 0)}
                history.append(rec)
                if log:
                    log(rec)
                if not opts.outer_backtrack:
                    u = u - du
                    continue
                # backtracking on ||F_x|| (the reading of the outer step): the first of
                # alpha = 1, 1/2, ... (at most min(ls_trials, 5)) with ||F(u')|| < outer_atol or
                # ||F_x(u')|| <= (1 - armijo alpha) ||F_x(u)||; the last trial is taken otherwise
                nFx, alpha = float(np.linalg.norm(Fx)), 1.0
                trials = min(opts.ls_trials, 5)
                for t in range(trials):
                    ut = u - alpha * du
                    if float(np.linalg.norm(self.F(ut, load))) < opts.outer_atol:
                        u = ut
                        break
                    Fxt, stt = self.evaluate(ut, load)
                    nt = float(np.linalg.norm(Fxt))
                    if (np.isfinite(nt) and nt <= (1.0 - opts.armijo * alpha) * nFx) or t == trials - 1:
                        u, cached = ut, (Fxt, stt)
                        break
                    alpha *= 0.5
            history.append({"load": load, "final_normF": nF})
        return u, history, time.perf_counter() - t0


# ----------------------------------------------------------------------------------------------
# GMRES(m) with modified Gram-Schmidt and Givens rotations (Section 3 settings)
# ----------------------------------------------------------------------------------------------

def gmres(A, b: np.ndarray, rtol: float, restart: int, maxit: int):
    """Solve A x = b from x = 0.  Returns (x, total iterations, final relative residual)."""
    x = np.zeros_like(b)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return x, 0, 0.0
    total = 0
    r = b.copy()
    rn = bn
    while total < maxit:
        V = [r / rn]
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = rn
        j = 0
        while j < restart and total < maxit:
            w = A(V[j])
            for i in range(j + 1):
                H[i, j] = float(np.dot(V[i], w))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0.0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            total += 1
            if abs(g[j]) <= rtol * bn:
                break
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
        for i in range(j):
            x = x + y[i] * V[i]
        r = b - A(x)
        rn = float(np.linalg.norm(r))
        if abs(g[j]) <= rtol * bn:
            break
    return x, total, rn / bn


# ----------------------------------------------------------------------------------------------
# the plain definition: global Newton on F(u) = 0 with a sparse direct solve
# ----------------------------------------------------------------------------------------------

def plain_newton(prob: Problem, tol: float = 1e-13, maxit: int = 50, load_steps: int = 1, u0=None):
    model = fem.Model(prob)
    N = prob.n_nodes * prob.ndof
    free = fem.free_mask(prob)
    u = np.zeros(N) if u0 is None else u0.copy()
    its_all = []
    for step in range(max(1, load_steps)):
        load = (step + 1) / max(1, load_steps)
        opts = Options(inner_atol=tol, inner_rtol=0.0, inner_maxit=maxit)

        def residual(x):
            full = u.copy()
            full[free] = x
            with np.errstate(invalid="ignore", divide="ignore"):
                F = fem.global_residual(model, full, load)
            return F[free], bool(np.all(np.isfinite(F)))

        def solve_jac(x, r):
            full = u.copy()
            full[free] = x
            J = fem.global_jacobian(model, full)[free][:, free].tocsc()
            return spla.spsolve(J, r)

        x, its, status, _, rn = newton(u[free], residual, solve_jac, opts)
        u[free] = x
        its_all.append((its, status, rn))
    return u, its_all
