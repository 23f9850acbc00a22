"""Mutation audit of the FP64 oracles (run by hand; pytest does not collect it).

Each entry plants one plausible mistake (a dropped term, a wrong sign, index
or factor, a misread rule) in a copy of ``oracle/`` and runs the CPU pin
suite (``tests/test_oracle_*.py``) against the copy.  A mistake that no pin
catches is a gap in the pins.  Entries marked ``equivalent`` change nothing
observable at the oracle's settings (the reason is given); they are listed
so that the audit's coverage is explicit.

    python tests/oracle_mutations.py [--jobs N] [--workdir DIR] [index ...]

Prints one line per mutation (CAUGHT with the first failing pin, or
SURVIVED) and exits 1 if a non-equivalent mutation survives.  The copies go
to DIR (default: the git-ignored .mutation_tmp of the repository, apart
from pytest's own temporary directory, which pytest empties at every start)
and are removed as each run ends; the tracked files are not modified.
"""
import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

BM, EDM, BB, BCD = "bm_oracle.py", "edm_oracle.py", "sparsa_oracle.py", "bcd_oracle.py"

# (oracle file, name, text, replacement, None or the reason it is equivalent)
MUTATIONS = [
    # index, codec, loss
    (BM, "index: csr2csc = csc2csr", "csr2csc[csc2csr] = np.arange(csc2csr.shape[0])", "csr2csc[:] = csc2csr", None),
    (BM, "index: no transpose when m > n", "transposed = m > n\n", "transposed = False\n", None),
    (BM, "codes: offset max", "return lo, (ix.val - lo)", "return hi, (ix.val - lo)", None),
    (BM, "codes: range 256", "if hi - lo > 255:", "if hi - lo > 256:", None),
    (BM, "loss: F with lam", "F = f + 0.5 * lam * (", "F = f + 1.0 * lam * (", None),
    (BM, "loss: gH without lam", "gH = R.T @ W + lam * H", "gH = R.T @ W", None),
    (BM, "residual: sign", "H[ix.col]) - ix.val", "H[ix.col]) + ix.val", None),
    (BM, "index: duplicates accepted", "        if np.any(same):\n            raise ValueError", "        if False:\n            raise ValueError", None),
    (BM, "index: CSC in CSR order", "csc2csr = np.lexsort((r_s, c_s))", "csc2csr = np.lexsort((c_s, r_s))", None),
    (BM, "codes: non-integers accepted", "if not np.all(v == np.rint(v)) or", "if not np.all(v == v) or", None),
    (BM, "generator: sine", "* np.cos(2.0 * math.pi * u[1::2])", "* np.sin(2.0 * math.pi * u[1::2])", None),
    (BM, "generator: 52-bit uniforms", "u = ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)",
     "u = ((z >> np.uint64(12)).astype(np.float64) + 1.0) * (2.0 ** -52)", None),
    (BM, "generator: key without the stream", "key = _mix64(np.array([(seed * _GAMMA + stream) & _M64]",
     "key = _mix64(np.array([(seed * _GAMMA) & _M64]", None),
    # orth (Eq. PUi, orth-W)
    (BM, "orth: one pass", "for pass_no in range(2):", "for pass_no in range(1):", None),
    (BM, "orth: L-image not projected", "                LMh = LMh - LF @ C\n", "                pass\n", None),
    (BM, "orth: T = E / lam", "T = E[:, good] / np.sqrt(lam_[good])", "T = E[:, good] / lam_[good]", None),
    (BM, "orth: no unit scaling", "Mh = M[:, keep] / s[keep]", "Mh = M[:, keep]", None),
    (BM, "orth: cap keeps the smallest", "good &= np.arange(lam_.shape[0]) < max_cols",
     "good &= np.arange(lam_.shape[0]) >= lam_.shape[0] - max_cols", None),
    # LmSVD (Algorithm 2)
    (BM, "lmsvd: memory p ignored", "blocks = [(Bnew, Lop(Bnew))] + blocks[:p]", "blocks = [(Bnew, Lop(Bnew))]", None),
    (BM, "lmsvd: stop relative to the smallest theta", "<= tol * max(theta[0], 1e-300)",
     "<= tol * max(theta[-1], 1e-300)", None),
    (BM, "lmsvd: smallest Ritz vectors", "Uh = Q @ V[:, :kk]\n        LUh = LQ @ V[:, :kk]\n        theta = th_all[:kk]",
     "Uh = Q @ V[:, -kk:]\n        LUh = LQ @ V[:, -kk:]\n        theta = th_all[-kk:]", None),
    (BM, "lmsvd: min_iter ignored", "if (it >= min_iter and theta_prev", "if (theta_prev",
     "at min_iter = 2 the test needs a previous theta, which exists only from the second step on"),
    (BM, "lmsvd: old blocks first", "Q = np.hstack([Bn, Q2])\n            LQ = np.hstack([LBn, LQ2])",
     "Q = np.hstack([Q2, Bn])\n            LQ = np.hstack([LQ2, LBn])",
     "the basis spans the same subspace, so the Rayleigh-Ritz values and vectors are the same"),
    # exact SVD, SVT, refactor
    (BM, "svt: half threshold", "sig = sh - thresh", "sig = sh - 0.5 * thresh", None),
    (BM, "svt: V not normalised", "V = (Bt @ Ut[:, :k_new]) / sh[:k_new]", "V = (Bt @ Ut[:, :k_new])", None),
    (BM, "svt: no square root in the refactor", "sq = np.sqrt(sig[:k_new])", "sq = sig[:k_new]", None),
    (BM, "svt: eps with thresholded values", "e2 = Zop.frob2() - float(np.sum(sh ** 2))",
     "e2 = Zop.frob2() - float(np.sum(sig[:k_new] ** 2))", None),
    (BM, "svt: truncated vector off by one", "u_tr = Uh @ Ut[:, k_new] if", "u_tr = Uh @ Ut[:, max(k_new - 1, 0)] if", None),
    (BM, "svt: cap at k_max - 1", "k_new = min(k_new, k_max)", "k_new = min(k_new, k_max - 1)", None),
    (BM, "Z: Z^T sign", "return self.H @ (self.W.T @ U) - self.alpha * (self.R.T @ U)",
     "return self.H @ (self.W.T @ U) + self.alpha * (self.R.T @ U)", None),
    (BM, "Z: Z sign", "return self.W @ (self.H.T @ Y) - self.alpha * (self.R @ Y)",
     "return self.W @ (self.H.T @ Y) + self.alpha * (self.R @ Y)", None),
    (BM, "Z: ||Z||^2 cross factor", "- 2.0 * self.alpha * (x @ self.r)", "- 1.0 * self.alpha * (x @ self.r)", None),
    (BM, "Z: ||Z||^2 alpha^2", "+ self.alpha ** 2 * (self.r @ self.r))", "+ self.alpha * (self.r @ self.r))", None),
    # PG step, safeguard, state
    (BM, "prox: threshold lam", "res = svt_refactor(Zop, Uh, lam * alpha, k_max)\n    return _advance",
     "res = svt_refactor(Zop, Uh, lam, k_max)\n    return _advance", None),
    (BM, "prox: Ritz cut on theta", "Uh = Uh[:, s > opt.ritz_rel * s[0]]", "Uh = Uh[:, theta > opt.ritz_rel * theta[0]]", None),
    (BM, "advance: psi halved off by one", "if res.k_new == warm_cols - 1 else", "if res.k_new == warm_cols else", None),
    (BM, "advance: U_{t-1} from this step", "U_prev2=st.U_prev, u=res.u_trunc", "U_prev2=res.U, u=res.u_trunc", None),
    (BM, "warm start: U_{t-1} after a BM phase",
     "second = st.W if (st.bm_changed or st.U_prev2 is None) else st.U_prev2",
     "second = st.U_prev2 if st.U_prev2 is not None else st.W", None),
    (BM, "warm start: xi not projected off U^", "        g = g - Uh0 @ (Uh0.T @ g)\n", "", None),
    (BM, "warm start: psi scales u_t", "col = ut + st.psi * g if st.u is not None else g",
     "col = st.psi * ut + g if st.u is not None else g", None),
    (BM, "warm start: cap k_max", "    cap = k_max + 1\n", "    cap = k_max\n", None),
    (BM, "init: sketch from the safeguard stream", "G = counter_normal(opt.seed, STREAM_INIT_SKETCH, m * k_init)",
     "G = counter_normal(opt.seed, STREAM_SAFEGUARD, m * k_init)", None),
    (BM, "init: sketch drawn column by column", ".reshape(k_init, m).T\n    Q, _ = orth(Zop.L(G)",
     ".reshape(m, k_init)\n    Q, _ = orth(Zop.L(G)", None),
    (BM, "solve: stop on the absolute change", "if abs(F_hist[-2] - F) / (1.0 + abs(F_hist[-2])) < tol:",
     "if abs(F_hist[-2] - F) < tol:", None),
    (BM, "warm start: and-trigger",
     "trig = (st.rank_hist[-1] == st.rank_hist[-2]) or (st.prev_warm_cols <= st.rank_hist[-1] + 1)",
     "trig = (st.rank_hist[-1] == st.rank_hist[-2]) and (st.prev_warm_cols <= st.rank_hist[-1] + 1)", None),
    # initial step (Eq. nys)
    (BM, "init: Z_{-1} sign", "Zop = ZOperator(ix, W0, H0, -ix.val.copy(), 1.0)",
     "Zop = ZOperator(ix, W0, H0, ix.val.copy(), 1.0)", None),
    (BM, "init: no Nystrom step", "Uh = Qh @ Ut[:, keep]", "Uh = Q[:, :int(np.sum(keep))]", None),
    (BM, "init: no pseudo-inverse cut", "Cpinv = (CE[:, cpos] / cw[cpos]) @ CE[:, cpos].T",
     "Cpinv = (CE / np.where(cw == 0, 1.0, cw)) @ CE.T",
     "orth(A G) already drops every direction whose eigenvalue is below about 1e-3 of the largest, "
     "so the cut never acts"),
    (BM, "init: Nystrom core transposed", "s2, Ut = eig_desc(Rh @ Cpinv @ Rh.T)", "s2, Ut = eig_desc(Rh.T @ Cpinv @ Rh)",
     "the core only orders the basis of ran(Q^) and feeds the Ritz cut, which never acts (above); "
     "the exact SVD that follows re-diagonalises within the same span"),
    # BM phase and Algorithm 1
    (BM, "bm: Fletcher-Reeves beta", "num = np.sum(gW * (gW - g_prev[0])) + np.sum(gH * (gH - g_prev[1]))",
     "num = np.sum(gW * gW) + np.sum(gH * gH)", None),
    (BM, "bm: no max(0, beta)", "beta = max(0.0, num / den)", "beta = num / den", None),
    (BM, "bm: -beta", "DW, DH = -gW + beta * DW, -gH + beta * DH", "DW, DH = -gW - beta * DW, -gH - beta * DH", None),
    (BM, "bm: quartic without lam in s^2", "+ 0.5 * lam * (np.sum(DW * DW) + np.sum(DH * DH))", "", None),
    (BM, "quartic: smallest root", "return cand[int(np.argmin(phi))]", "return cand[1] if len(cand) > 1 else 0.0", None),
    (BM, "solve: PG step before the BM phase",
     "        st, _ = bm_phase(ix, st, lam, opt.bm_epochs)\n        for _ in range(opt.pg_steps):\n"
     "            st, info = prox_step(ix, st, lam, k_max, opt)\n            eps_hist.append(info.eps)\n"
     "            its.append(info.lmsvd_iters)\n",
     "        for _ in range(opt.pg_steps):\n            st, info = prox_step(ix, st, lam, k_max, opt)\n"
     "            eps_hist.append(info.eps)\n            its.append(info.lmsvd_iters)\n"
     "        st, _ = bm_phase(ix, st, lam, opt.bm_epochs)\n", None),
    (BM, "edm lambda: sign", "return -10.0 * math.sqrt(n) / float(", "return 10.0 * math.sqrt(n) / float(", None),
    (BM, "edm lambda: sqrt(n) / 10", "return -10.0 * math.sqrt(n) / float(np.sum(np.asarray(d, dtype=np.float64) ** 2))",
     "return -math.sqrt(n) / 10.0", None),
    # distance-geometry QSDP
    (EDM, "edm: residual sign of d^2", "return np.sum(diff * diff, axis=1) - d * d",
     "return np.sum(diff * diff, axis=1) + d * d", None),
    (EDM, "edm: objective lam / 2", "return 0.5 * float(np.sum(w * r * r)) + lam * float(np.sum(V * V))",
     "return 0.5 * float(np.sum(w * r * r)) + 0.5 * lam * float(np.sum(V * V))", None),
    (EDM, "edm: Laplacian sign", "np.add.at(out, j, -D)", "np.add.at(out, j, D)", None),
    (EDM, "edm: gradient factor", "return 2.0 * laplacian_apply(V.shape[0], i, j, w * r, V) + 2.0 * lam * V",
     "return 1.0 * laplacian_apply(V.shape[0], i, j, w * r, V) + 2.0 * lam * V", None),
    (EDM, "edm: Lipschitz diagonal", "return float(np.max(4.0 * w + sw", "return float(np.max(2.0 * w + sw", None),
    (EDM, "edm: centring over rows", "return U - U.mean(axis=0, keepdims=True)", "return U - U.mean(axis=1, keepdims=True)", None),
    (EDM, "edm: Fletcher-Reeves beta", "float(np.sum(g * (g - g_prev)))", "float(np.sum(g * g))", None),
    (EDM, "edm: Z without alpha", "c = alpha * w * r", "c = w * r", None),
    (EDM, "edm: Z shift sign of lam J", "- self.alpha * self.lam * center(U))", "+ self.alpha * self.lam * center(U))", None),
    (EDM, "edm: shift not removed", "return Uh[:, :kk], theta[:kk] - Zop.sigma, iters", "return Uh[:, :kk], theta[:kk], iters", None),
    (EDM, "edm: shift by sigma I", "return self.z(U) + self.sigma * center(U)", "return self.z(U) + self.sigma * U", None),
    (EDM, "edm: shift half the bound", "sigma = 2.0 * float(np.max(rowabs))", "sigma = 1.0 * float(np.max(rowabs))", None),
    (EDM, "edm: factor mu not sqrt(mu)", "Vn = U[:, pos] * np.sqrt(mu[pos])", "Vn = U[:, pos] * mu[pos]", None),
    (EDM, "edm: rank rule growth n / 10", "k_next = min(k_max, k_eig + n // 20)", "k_next = min(k_max, k_eig + n // 10)", None),
    (EDM, "edm: rank rule keeps k when truncated", "k_next = max(1, rank)", "k_next = max(1, k_eig)", None),
    (EDM, "edm: warm start not centred", "Q, _ = O.orth(center(M), max_cols=k)", "Q, _ = O.orth(M, max_cols=k)",
     "U_t and V already lie in ker(e^T), so the centring only removes rounding, and with the shift sigma J a "
     "component along e decays (eigenvalue 0) and is never among the leading pairs"),
    (EDM, "edm: initial rank 0.1 n", "k0 = max(1, min(100, int(0.15 * n), k_max))", "k0 = max(1, min(100, int(0.1 * n), k_max))", None),
    (EDM, "edm: step 1.99 / L", "alpha = 1.0 / lipschitz(n, i, j, w)\n    st, _ = init_step",
     "alpha = 1.99 / lipschitz(n, i, j, w)\n    st, _ = init_step", None),
    (EDM, "edm: PG step before the BM phase",
     "        V, _ = bm_phase(st.V, i, j, d, w, lam, opt.bm_epochs)\n        st = EdmState(V=V, U=st.U, k_eig=st.k_eig, t=st.t)\n"
     "        st, info = prox_step(st, i, j, d, w, lam, alpha, k_max, opt)\n",
     "        st, info = prox_step(st, i, j, d, w, lam, alpha, k_max, opt)\n"
     "        V, _ = bm_phase(st.V, i, j, d, w, lam, opt.bm_epochs)\n        st = EdmState(V=V, U=st.U, k_eig=st.k_eig, t=st.t)\n",
     None),
    (EDM, "edm: fill columns from stream t", "G = O.counter_normal(seed, STREAM_EDM_FILL + t, n * extra)",
     "G = O.counter_normal(seed, t, n * extra)", None),
    (EDM, "edm: initial start not centred", "U, mu, iters = top_eigpairs(Zop, center(G), k0, opt)",
     "U, mu, iters = top_eigpairs(Zop, G, k0, opt)",
     "with the shift sigma J, e carries the eigenvalue 0, the bottom of the positive semidefinite shifted "
     "spectrum: a start component along e decays and is never among the leading pairs"),
    (EDM, "edm dense reference: off-diagonal gradient doubled", "    np.add.at(G, (i, j), -c)\n", "    np.add.at(G, (i, j), -2.0 * c)\n", None),
    (EDM, "edm dense reference: solve steps with lam / 2",
     "Xn = dense_project(Y - alpha * (dense_grad_f(Y, i, j, d, w) + lam * np.eye(n)))",
     "Xn = dense_project(Y - alpha * (dense_grad_f(Y, i, j, d, w) + 0.5 * lam * np.eye(n)))", None),
    # SpaRSA step rule
    (BB, "bb: trace cross factor", "return t11 + t00 - 2.0 * t01", "return t11 + t00 - t01", None),
    (BB, "bb: nuclear norm without sqrt", "return float(np.sum(np.sqrt(np.maximum(ev, 0.0))))",
     "return float(np.sum(np.maximum(ev, 0.0)))", None),
    (BB, "bb: curvature instead of step", "a = o.alpha_max if den <= 0 else num / den",
     "a = o.alpha_max if den <= 0 else den / num", None),
    (BB, "bb: no clipping", "return max(o.alpha_min, min(o.alpha_max, a))", "return a", None),
    (BB, "bb: first trial already reduced", "a = a0 * o.beta ** i", "a = a0 * o.beta ** (i + 1)", None),
    (BB, "bb: Eq. back with 2 alpha", "back = f1 <= f + lin + o.delta / a * d2", "back = f1 <= f + lin + o.delta / (2.0 * a) * d2", None),
    (BB, "bb: Q with d2 / alpha", "Q = lin + d2 / (2.0 * a) +", "Q = lin + d2 / a +", None),
    (BB, "bb: decrease sign", "dec = F1 <= F0 + o.delta * Q", "dec = F1 <= F0 - o.delta * Q", None),
    (BB, "bb: previous point after the step", "return st1, info, bb, BbPoint(st.W.copy(), st.H.copy(), r)",
     "return st1, info, bb, BbPoint(st1.W.copy(), st1.H.copy(), O.residual(ix, st1.W, st1.H))", None),
    (BB, "bb: first step alpha 1", "a0 = bb_alpha(st.W, st.H, r, prev, o, opt.alpha)", "a0 = bb_alpha(st.W, st.H, r, prev, o, 1.0)", None),
    (BB, "bb: exhausted search keeps the first trial", "        out = (st1, info, BbInfo(a0, a, i, 1 if back else (2 if dec else 0)))",
     "        out = out or (st1, info, BbInfo(a0, a, i, 1 if back else (2 if dec else 0)))", None),
    (BB, "bb: solve forgets the previous point", "st, info, bb, prev = prox_step_bb(ix, st, lam, k_max, opt, o, prev)",
     "st, info, bb, _ = prox_step_bb(ix, st, lam, k_max, opt, o, prev)", None),
    # column-block coordinate descent
    (BCD, "bcd: block gradient without lam", "gw = R @ h + lam * w", "gw = R @ h", None),
    (BCD, "bcd: b without the H term", "b = dw[ri] * h[cj] + w[ri] * dh[cj]", "b = dw[ri] * h[cj]", None),
    (BCD, "bcd: quartic without lam in s^2", "+ 0.5 * lam * (float(dw @ dw) + float(dh @ dh)),", ",", None),
    (BCD, "bcd: residual update without s^2", "r = r + s * b + s * s * cc", "r = r + s * b", None),
    (BCD, "bcd: phase reports the first block", "F.append(tr[-1] if tr else", "F.append(tr[0] if tr else", None),
    (BCD, "bcd: blocks in reverse order", "for c in range(W.shape[1]):", "for c in reversed(range(W.shape[1])):", None),
]


def _copy_tree(dst):
    for sub in ("oracle", "synth"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(dst, sub), ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f.endswith(".py") and not f.startswith("test_gpu_") and f != os.path.basename(__file__):
            shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))


def run_one(idx, workdir):
    fname, name, old, new, _ = MUTATIONS[idx]
    d = os.path.join(workdir, str(idx))
    if os.path.exists(d):
        shutil.rmtree(d)
    os.makedirs(d)
    _copy_tree(d)
    p = os.path.join(d, "oracle", fname)
    with open(p) as f:
        src = f.read()
    if src.count(old) != 1:
        return f"PATTERN x{src.count(old)}"
    with open(p, "w") as f:
        f.write(src.replace(old, new))
    tests = sorted(os.path.join("tests", t) for t in os.listdir(os.path.join(d, "tests")) if t.startswith("test_oracle_"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *tests],
                       cwd=d, capture_output=True, text=True, timeout=1800,
                       env={**os.environ, "OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1"})
    shutil.rmtree(d, ignore_errors=True)
    if r.returncode == 0:
        return "SURVIVED"
    failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED") or ln.startswith("ERROR")]
    return "CAUGHT " + (failed[0].split(" - ")[0].replace("FAILED ", "") if failed else "(collection)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--workdir", default=None)
    ap.add_argument("which", nargs="*", type=int)
    a = ap.parse_args()
    work = a.workdir or os.path.join(ROOT, ".mutation_tmp")
    os.makedirs(work, exist_ok=True)
    idx = a.which or list(range(len(MUTATIONS)))
    bad_idx = [i for i in idx if not 0 <= i < len(MUTATIONS)]
    if bad_idx:
        ap.error(f"no mutation {bad_idx}: indices run from 0 to {len(MUTATIONS) - 1}")
    with cf.ThreadPoolExecutor(a.jobs) as ex:
        res = dict(zip(idx, ex.map(lambda i: run_one(i, work), idx)))
    bad = 0
    for i in idx:
        fname, name, _, _, eq = MUTATIONS[i]
        line = f"{i:3d} {fname:17s} {name:45s} {res[i]}"
        if eq is not None:
            line += f"  [equivalent: {eq}]"
        elif not res[i].startswith("CAUGHT"):
            bad += 1
        print(line, flush=True)
    caught = sum(res[i].startswith("CAUGHT") for i in idx)
    n_eq = sum(MUTATIONS[i][4] is not None for i in idx)
    print(f"{caught} of {len(idx)} caught; {n_eq} marked equivalent; {bad} non-equivalent not caught")
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
