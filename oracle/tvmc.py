"""otVMC evaluation, regularised solve and Stratonovich step, in plain FP64.

Test infrastructure (oracle side): only tests, the smoke check and the CPU baseline of the
benchmark use this module.  Nothing here is blocked, fused or reordered beyond the
definitions; numpy library routines (matmul, Cholesky, eigh) serve as steps.

One *evaluation* at parameters theta follows the otVMC procedure (text after Eq. 9):
  1. configurations x drawn from |psi_theta(x)|^2 (Metropolis, or exact weights),
  2. local operators O_k(x), local effective energy E_eff(x) and local noises B^n(x)
     (definitions after Eq. 8, effective Hamiltonian Eq. 5),
  3. S, F, N^n as covariances over the samples (definitions after Eq. 8),
  4. D = -i F dt + sum_n N^n dW_n (otVMC procedure paragraph),
  5. delta solving (S + eps I) delta = D (diagonal shift) or the SNR-filtered
     eigen-pseudo-inverse of the same paragraph.
A trajectory step is the predictor-corrector scheme of App. C applied to theta.

Readings where the paper is silent (each one listed in the design notes):
* <L_n + L_n^+> inside H_eff is estimated from the same samples as the real part of the
  mean of the local estimator of L_n + L_n^+; exact under exact weights.
* The c-number terms of H_eff (Eq. 5, <L+L^+>^2 - 1/2<L^2 + 2L^+L + L^+2>) are dropped:
  they shift E_eff by a constant, which cancels in F and N^n.
* Jump operators: decay L = sqrt(kappa) s^-_j and dephasing L = sqrt(gamma) sz_j, with
  local estimators
     decay:    B = sqrt(kappa) [sigma_j = -1] r_j,  (L^+L)_loc = kappa (1 + sigma_j)/2,
               (L^2)_loc = 0,  (L + L^+)_loc = sqrt(kappa) r_j
     dephase:  B = sqrt(gamma) sigma_j,  (L^+L)_loc = (L^2)_loc = gamma,
               (L + L^+)_loc = 2 sqrt(gamma) sigma_j
  and E_H(x) = sum_{i<j} J_ij sigma_i sigma_j + h sum_j r_j(x).
"""
import numpy as np
import scipy.linalg

from .philox import proposal_draws


# ----------------------------------------------------------------------- local estimators

def local_terms(model, ans, theta, sig):
    """Per-sample quantities that do not depend on <L+L^+>.

    Returns dict with r (Ns, N) flip ratios, EH (Ns,), B (Ns, n_ops), LdL (Ns, n_ops),
    L2 (Ns, n_ops), LpLd (Ns, n_ops) local estimators of L^+L, L^2, L + L^+.
    """
    s = sig.astype(np.float64)
    r = np.exp(ans.log_flip_ratios(theta, sig))
    EH = 0.5 * np.einsum("xi,ij,xj->x", s, model.J, s) + model.h * r.sum(axis=1)
    ops = model.jump_ops()
    ns = sig.shape[0]
    B = np.zeros((ns, len(ops)), complex)
    LdL = np.zeros((ns, len(ops)), complex)
    L2 = np.zeros((ns, len(ops)), complex)
    LpLd = np.zeros((ns, len(ops)), complex)
    for n, (kind, j, rate) in enumerate(ops):
        if kind == "decay":
            B[:, n] = np.sqrt(rate) * (s[:, j] < 0) * r[:, j]
            LdL[:, n] = rate * (1 + s[:, j]) / 2
            L2[:, n] = 0.0
            LpLd[:, n] = np.sqrt(rate) * r[:, j]
        else:
            B[:, n] = np.sqrt(rate) * s[:, j]
            LdL[:, n] = rate
            L2[:, n] = rate
            LpLd[:, n] = 2 * np.sqrt(rate) * s[:, j]
    return dict(r=r, EH=EH, B=B, LdL=LdL, L2=L2, LpLd=LpLd)


def effective_energy(terms, lpl):
    """E_eff(x) = E_H - i/2 sum_n [(L^+L)_loc - 2 <L+L^+> B^n + (L^2)_loc]  (Eq. 5)."""
    bracket = terms["LdL"] - 2.0 * lpl[None, :] * terms["B"] + terms["L2"]
    return terms["EH"] - 0.5j * bracket.sum(axis=1)


def effective_energy_linear(terms):
    """E_eff^lin(x) = <x|H_lin|psi>/psi(x), H_lin = H - i/2 sum_n (L^+L + L^2) (linear SSE, App. B)."""
    return terms["EH"] - 0.5j * (terms["LdL"] + terms["L2"]).sum(axis=1)


def expectation(w, X):
    """sum_x w(x) X(x, ...) with weights summing to one (MC: 1/Ns; exact: |psi|^2/Z)."""
    return np.tensordot(w, X, axes=(0, 0))


def covariance(w, A, B):
    """<A^* B> - <A^*><B> over the rows (definitions of S, F, N^n after Eq. 8)."""
    Ac = A.conj()
    return Ac.T @ (w[:, None] * B) - np.outer(expectation(w, Ac), expectation(w, B))


def evaluate(model, ans, theta, sig, w, dW, dt, with_S=True, linear=False):
    """S, F, N^n and D at theta from configurations sig with weights w.

    D = -i F dt + sum_n N^n dW_n (otVMC procedure paragraph, hbar = 1).  with_S=False skips
    the P x P matrix S (S is None then), for parameter counts where only the push-through
    solve below is affordable.  linear=True takes the linear SSE's local effective energy
    E_eff^lin in place of E_eff (App. B), so that F is F^lin.
    """
    terms = local_terms(model, ans, theta, sig)
    lpl = expectation(w, terms["LpLd"]).real
    E = effective_energy_linear(terms) if linear else effective_energy(terms, lpl)
    O = ans.O(theta, sig)
    S = covariance(w, O, O) if with_S else None
    F = covariance(w, O, E[:, None])[:, 0]
    N = covariance(w, O, terms["B"])
    D = -1j * F * dt + N @ np.asarray(dW, dtype=np.float64)
    return dict(S=S, F=F, N=N, D=D, E=E, lpl=lpl, O=O, terms=terms)


def mc_weights(ns):
    return np.full(ns, 1.0 / ns)


def all_configs(n):
    x = np.arange(2 ** n)[:, None]
    return np.where((x >> np.arange(n)[None, :]) & 1, 1, -1).astype(np.int8)


def exact_weights(ans, theta, sig):
    lp = ans.logpsi(theta, sig)
    p = np.exp(2 * (lp.real - lp.real.max()))
    return p / p.sum()


def evaluate_enumeration(model, ans, theta, dW, dt):
    """Evaluation with exact expectations over all 2^N configurations (N <= 12)."""
    sig = all_configs(ans.n)
    return evaluate(model, ans, theta, sig, exact_weights(ans, theta, sig), dW, dt)


# ------------------------------------------------------------------------------- solves

def solve_shift(S, D, eps):
    """(S + eps I) delta = D by Cholesky (diagonal-shift regularisation)."""
    A = S + eps * np.eye(S.shape[0])
    c = scipy.linalg.cho_factor(A, lower=True)
    return scipy.linalg.cho_solve(c, D)


def solve_shift_push(O, v, w, eps):
    """The same delta as solve_shift(S, D, eps), through a system of size Ns.

    With A = W^(1/2) O_c (rows scaled by sqrt(w), O_c centred) and b = W^(1/2) v_c, the
    covariances are S = A^+ A and D = A^+ b, and (A^+ A + eps I)^-1 A^+ = A^+ (A A^+ + eps I)^-1
    (push-through identity), so delta = A^+ (A A^+ + eps I)^-1 b: a Cholesky of Ns x Ns instead
    of P x P.  For MC weights A A^+ = O_c O_c^+ / Ns.
    """
    sw = np.sqrt(np.asarray(w, dtype=np.float64))
    A = sw[:, None] * (O - expectation(w, O)[None, :])
    b = sw * (v - expectation(w, v))
    K = A @ A.conj().T + eps * np.eye(A.shape[0])
    c = scipy.linalg.cho_factor(K, lower=True)
    return A.conj().T @ scipy.linalg.cho_solve(c, b)


def solve_snr(S, D, O, v, w, snr_thresh=4.0, eps_svd=1e-12):
    """SNR-regularised pseudo-inverse in the eigenbasis of S (otVMC procedure paragraph).

    S = V diag(lam) V^+, rho = V^+ D.  Per-sample contributions Q_k(x) = (V^+ O_c^*(x))_k
    v_c(x) average to rho_k; SNR_k = |rho_k| / sqrt(Var Q_k / Ns).  Each inverse
    eigenvalue is damped by 1/(1 + (snr_thresh/SNR_k)^6) and 1/(1 + (eps_svd lam_max/lam_k)^6).
    The filter shape is a reading of the cited regularisation, not printed in the paper:
    parity unpinned beyond its limit (thresholds -> 0 gives the plain pseudo-inverse).
    MC weights only (w = 1/Ns).
    """
    lam, V = np.linalg.eigh(S)
    rho = V.conj().T @ D
    Oc = O - expectation(w, O)[None, :]
    vc = v - expectation(w, v)
    Q = (Oc.conj() @ V) * vc[:, None]          # Q[x, k]
    ns = O.shape[0]
    var = (np.abs(Q - Q.mean(axis=0)) ** 2).mean(axis=0)
    snr = np.abs(rho) / np.sqrt(var / ns + 1e-300)
    lam_max = lam.max()
    with np.errstate(divide="ignore", over="ignore"):
        f_snr = 1.0 / (1.0 + (snr_thresh / snr) ** 6)
        f_svd = 1.0 / (1.0 + (eps_svd * lam_max / np.maximum(lam, 1e-300)) ** 6)
        inv = np.where(lam > 0, f_snr * f_svd / np.maximum(lam, 1e-300), 0.0)
    return V @ (inv * rho)


def log_norm_increment(ev, w, dW, dt):
    """Increment of ln Q over one step of the linear SSE (normalisation SDE of App. B, dQ =
    Q (2 Im<E_eff^lin> dt + 2 sum_n Re<B^n> o dW_n), Stratonovich, so d ln Q is the bracket)."""
    Emean = expectation(w, ev["E"])
    Bmean = expectation(w, ev["terms"]["B"])
    return 2.0 * Emean.imag * dt + 2.0 * float(np.dot(Bmean.real, np.asarray(dW, dtype=np.float64)))


def local_v(ev, dW, dt):
    """v(x) = -i dt E_eff(x) + sum_n dW_n B^n(x), so that D = Cov(O^*, v)."""
    return -1j * dt * ev["E"] + ev["terms"]["B"] @ np.asarray(dW, dtype=np.float64)


# -------------------------------------------------------------------------------- sampler

def metropolis(ans, theta, sig, seed, traj_id, eval_index, n_sweep, chain_ids=None):
    """Single-spin-flip Metropolis on |psi_theta|^2, one chain per row of sig.

    n_sweep * N proposals per chain; proposal p flips the site drawn for it and is
    accepted iff u < |psi(x')/psi(x)|^2 = exp(2 Re log r_site).  Plain FP64: the log
    ratio is recomputed from scratch for every proposal.  Row r of sig is chain r, or chain
    chain_ids[r] when given (its random stream is keyed by the chain id).
    """
    sig = np.array(sig, dtype=np.int8, copy=True)
    nc, n = sig.shape
    rows = np.arange(nc)
    accepted = np.zeros(nc, dtype=np.int64)
    for p in range(n_sweep * n):
        site, u = proposal_draws(seed, traj_id, nc, eval_index, p, n, chain_ids)
        lr = log_flip_ratio_at(ans, theta, sig, site)
        acc = u < np.exp(2.0 * lr.real)
        sig[rows[acc], site[acc]] *= -1
        accepted += acc
    return sig, accepted


def log_flip_ratio_at(ans, theta, sig, site):
    """log r_site(x) for one site per chain (same formulas as the ansatz classes)."""
    s = sig.astype(np.float64)
    rows = np.arange(sig.shape[0])
    if ans.kind == "jastrow":
        a, eta = ans.split(theta)
        field = a[site] + np.einsum("xk,xk->x", eta[site], s)
        return -2.0 * s[rows, site] * field
    a, b, W = ans.split(theta)
    from .ansatz import log2cosh
    g = b[None, :] + s @ W
    sj = s[rows, site]
    g1 = g - 2.0 * sj[:, None] * W[site]
    return -2.0 * a[site] * sj + (log2cosh(g1) - log2cosh(g)).sum(axis=1)


# ----------------------------------------------------------------------------- SDE steps

def sde_step(theta, increment, scheme):
    """One step of App. C: predictor X-bar = X + delta(X); trapezoidal (Heun) corrector
    X' = X + (delta(X) + delta(X-bar))/2, or midpoint X' = X + delta((X + X-bar)/2).

    increment(theta, stage) returns delta = A dt + B dW at theta, with the same dW for both
    stages.  Returns (theta', delta_predictor, delta_corrector).
    """
    d0 = increment(theta, 0)
    pred = theta + d0
    if scheme == "heun":
        d1 = increment(pred, 1)
        return theta + 0.5 * (d0 + d1), d0, d1
    if scheme == "midpoint":
        d1 = increment(0.5 * (theta + pred), 1)
        return theta + d1, d0, d1
    raise ValueError(scheme)
