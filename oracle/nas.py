"""Algorithm 3 (augmented subspace method) and the direct SCF (oracle).

Test infrastructure: plain FP64 NumPy/SciPy, written from the paper's Sec. 3.3.

One augmented-subspace step (Algorithm 3 body):
  1. N shifted linear boundary value problems (Algorithm 3, step 1)
       (H~ u^_i, v) = (lambda_i + mu)(psi_i, v),  H~ = -1/2 Lap + V_ext + mu + V_Har + V_xc,
     i.e. (K/2 + M_Vext + M_(VH+Vxc)(rho) + mu M) u^_i = (lambda_i + mu) M psi_i.
  2. the small Kohn-Sham problem in S_H + span{u^_i}, solved by SCF; each SCF
     iteration solves F_A U = lambda F_B U with the 2x2 block
     matrices of Sec. 3.3:
       F_A = [[A_H, b_H], [b_H^T, beta]],   F_B = [[B_H, c_H], [c_H^T, gamma]],
       A_H = I^T A_h I, b_H = I^T A_h U^, beta = U^T A_h U^,
       c_H = I^T M U^, gamma = U^T M U^, A_h = A^L + A^NL.
  3. density update rho = sum_i f_i psi_i^2.

Readings (where the paper is silent, ambiguous or garbled):
  * density: rho = sum_i f_i |psi_i|^2 with occupations f_i (2 per orbital,
    closed shell); the printed update sum_i psi_i has neither square nor f_i.
  * F_A is built from H (no mu): the shift only moves the eigenvalues of the
    small problem by mu, because F_B is the exact Gram matrix of the basis.
  * B_H = I^T M_h I on the fine mesh (the paper assembles it on T_H), so that
    F_B is the exact Gram matrix of {I phi_a} U {u^_i} and the small problem is
    a Rayleigh-Ritz projection within S_h.
  * inner SCF: iterate to ||rho_out - rho_in||_0 < tol (cap max_inner), with
    Anderson mixing; the state carried to the next step is (Lambda, Psi) of the
    last small eigenproblem and the density rho_in that defined its potential.
    H~ in the next step uses that same rho_in.
  * outer stop: ||rho^(l) - rho^(l-1)||_0 < tol_scf with rho^(l) = sum f psi^2,
    or l > max_outer.
  * energy (Sec. 3.1): E = sum_i f_i lambda_i - int (V_H/2 + V_xc) rho
    + E_xc + E_nn, all density-dependent terms at the density rho_in of the
    potential.
  * basis of the augmented space: before the blocks of F_A, F_B are formed, the
    u^_i are replaced by an M-orthonormal basis of their M-orthogonal
    complement to I S_H (u^ <- u^ - I B_H^-1 I^T M u^, then u^ <- u^ L^-T with
    L L^T = u^T M u^).  This spans the same augmented subspace S_H + span{u^_i},
    so the Ritz pairs of the small problem are unchanged; it is needed because with the
    experiments' large mu each u^_i differs from a coarse-space function only
    by O(1/mu), which makes F_B in the printed basis nearly singular
    (condition number ~1e11 on the 8-nucleus workload).
  * initial guess: the self-consistent solution in the coarse space alone
    (S_H carried to the fine mesh by I), from rho = 0, by the same inner SCF.
  * mu defaults to the experiments' 8 M sum_k Z_k^2.
  * Anderson restart (option, off by default): in the inner SCF a density
    residual above anderson_restart x the best residual so far clears the
    mixing history.
  * occupations: the given f_i (closed shell), or, with smearing kT > 0,
    Fermi-Dirac f_i = 2/(1 + exp((lambda_i - eF)/kT)) with sum f_i equal to the
    electron count, recomputed after every small eigensolve; the energy is
    then the free energy E - kT S, S = -2 sum [g ln g + (1-g) ln(1-g)], g = f/2.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem, lda, hartree, transfer
from .anderson import Anderson
from .linalg import solve_spd

POT_COULOMB, POT_SMOOTHED, POT_HARMONIC = 0, 1, 2


def external_potential(inst, xq):
    """V_ext at points xq [..., 3] (Sec. 2: -sum_k Z_k/|x - R_k|)."""
    V = np.zeros(xq.shape[:-1])
    if inst.potential == POT_HARMONIC:
        return 0.5 * inst.omega ** 2 * np.sum(xq ** 2, axis=-1)
    for Rk, Zk in zip(inst.R, inst.Z):
        r2 = np.sum((xq - Rk) ** 2, axis=-1)
        if inst.potential == POT_SMOOTHED:
            V -= Zk / np.sqrt(r2 + inst.smooth_a ** 2)
        else:
            V -= Zk / np.sqrt(r2)
    return V


def dvext_dparams(inst, xq):
    """d V_ext / d(R_k, Z_k) at points xq: array [M, 4, ...] (x, y, z, Z)."""
    out = np.zeros((len(inst.Z), 4) + xq.shape[:-1])
    for k, (Rk, Zk) in enumerate(zip(inst.R, inst.Z)):
        d = xq - Rk
        r2 = np.sum(d * d, axis=-1)
        if inst.potential == POT_SMOOTHED:
            r2 = r2 + inst.smooth_a ** 2
        inv = 1.0 / np.sqrt(r2)
        # V = -Z (r2)^(-1/2): dV/dR = -Z (x - R) r2^(-3/2); dV/dZ = -r2^(-1/2)
        for c in range(3):
            out[k, c] = -Zk * d[..., c] * inv ** 3
        out[k, 3] = -inv
    return out


def nuclear_repulsion_grad(inst):
    """d E_nn / d(R_k, Z_k): [M, 4]."""
    g = np.zeros((len(inst.Z), 4))
    for j in range(len(inst.Z)):
        for k in range(len(inst.Z)):
            if j == k:
                continue
            d = inst.R[k] - inst.R[j]
            r = np.linalg.norm(d)
            g[k, :3] -= inst.Z[j] * inst.Z[k] * d / r ** 3
            g[k, 3] += inst.Z[j] / r
    return g


def nuclear_repulsion(inst):
    """E_nn = sum_{k<j} Z_j Z_k / |R_j - R_k| (Sec. 3.1)."""
    E = 0.0
    for j in range(len(inst.Z)):
        for k in range(j):
            E += inst.Z[j] * inst.Z[k] / np.linalg.norm(inst.R[j] - inst.R[k])
    return E


def fermi_dirac(lam, n_el, kT):
    """Occupations 2/(1 + exp((lam - eF)/kT)) summing to n_el, and -kT S.

    eF is found by bisection on the (increasing) electron count; S is the
    entropy of independent spin-degenerate levels, -2 sum [g ln g + (1-g) ln(1-g)]
    with g = f/2.
    """
    lam = np.asarray(lam, dtype=np.float64)
    if not n_el < 2.0 * len(lam):
        raise ValueError("smearing needs more orbitals than n_el / 2")

    def occ(eF):
        with np.errstate(over="ignore"):      # exp -> inf gives the exact limit f = 0
            return 2.0 / (1.0 + np.exp((lam - eF) / kT))

    def count(eF):
        return float(np.sum(occ(eF)))

    lo, hi = lam.min() - 50.0 * kT - 1.0, lam.max() + 50.0 * kT + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if count(mid) < n_el:
            lo = mid
        else:
            hi = mid
    eF = 0.5 * (lo + hi)
    f = occ(eF)
    g = 0.5 * f
    inside = (g > 0.0) & (g < 1.0)
    S = -2.0 * float(np.sum(g[inside] * np.log(g[inside]) + (1.0 - g[inside]) * np.log1p(-g[inside])))
    return f, -kT * S


def default_mu(inst):
    return 8.0 * len(inst.Z) * float(np.sum(np.asarray(inst.Z) ** 2))


@dataclass
class State:
    lam: np.ndarray            # [N] eigenvalues
    Psi: np.ndarray            # [n, N] fine interior values of the orbitals
    rho_in: np.ndarray         # [ne, nq] density defining the potential
    rho_out: np.ndarray        # [ne, nq] sum f psi^2
    VH: np.ndarray             # [nnode] Hartree potential of rho_in (nodal)
    occ: np.ndarray = None     # [N] occupations of these orbitals
    minus_TS: float = 0.0      # -kT S of the occupations (smearing)
    n_inner: int = 0
    inner_res: float = 0.0
    inner_converged: bool = True
    info: dict = field(default_factory=dict)


class Problem:
    """Fine/coarse spaces, fixed matrices and the transfer of one instance."""

    def __init__(self, inst, with_transfer=True):
        self.inst = inst
        self.fine = fem.Space(inst.fine_xyz, inst.fine_tet, inst.order)
        self.coarse = fem.Space(inst.coarse_xyz, inst.coarse_tet, 1)
        f = self.fine
        Kf = f.assemble_full("K")
        Mf = f.assemble_full("M")
        self.K = f.interior(Kf)
        self.K_IB = f.interior_boundary(Kf)
        self.M = f.interior(Mf)
        self.vext_q = external_potential(inst, f.xq)
        self.Mvext = f.interior(f.assemble_full("M", coef=self.vext_q))
        self.AL = (0.5 * self.K + self.Mvext).tocsr()   # A_h^L of Sec. 3.3, without mu
        self.mu = default_mu(inst) if inst.mu is None else float(inst.mu)
        self.occ = np.asarray(inst.occ, dtype=np.float64)
        self.N = len(self.occ)
        self.Enn = nuclear_repulsion(inst)
        if with_transfer:
            self.I, self.I_elem, self.I_W, self.I_C = transfer.build_transfer(f, self.coarse)
            self.B_H = (self.I.T @ self.M @ self.I).toarray()
            self.A_HL = (self.I.T @ self.AL @ self.I).toarray()
            self.B_H_chol = sla.cho_factor(self.B_H, lower=True)

    # ------------------------------------------------------------ potentials
    def nonlinear(self, rho_q, VH_guess=None):
        """(V_H nodal, V_H at quad points, eps_xc, v_xc) for density rho_q."""
        f = self.fine
        if self.inst.hartree:
            x0 = None if VH_guess is None else VH_guess[f.interior_nodes]
            VH = hartree.hartree(f, self.K, self.K_IB, rho_q, tol=self.inst.tol_poisson * 1e-1,
                                 x0=x0)
        else:
            VH = np.zeros(f.nnode)
        VHq = f.at_quad(VH)
        if self.inst.xc:
            eps, vxc = lda.lda(rho_q)
        else:
            eps = np.zeros_like(rho_q)
            vxc = np.zeros_like(rho_q)
        return VH, VHq, eps, vxc

    def A_NL(self, VHq, vxc):
        """A_h^NL of Sec. 3.3: ((V_Har + V_xc) phi_i, phi_j) on the interior."""
        return self.fine.interior(self.fine.assemble_full("M", coef=VHq + vxc))

    def density(self, Psi, occ=None):
        """rho = sum_i f_i psi_i^2 at quadrature points."""
        occ = self.occ if occ is None else occ
        Pq = self.fine.at_quad(self.fine.to_nodes(Psi))   # [ne, nq, N]
        return np.einsum("eqn,n->eq", Pq * Pq, occ)

    def occupations(self, lam):
        """(f, -kT S): the given occupations, or Fermi-Dirac ones with smearing."""
        kT = float(getattr(self.inst, "smearing", 0.0))
        if kT > 0.0:
            return fermi_dirac(lam, float(np.sum(self.occ)), kT)
        return self.occ, 0.0

    def norm0(self, f_q):
        return float(np.sqrt(np.sum(self.fine.Wq * f_q * f_q)))

    # ------------------------------------------------------------ small problem
    def small_blocks(self, A, Uhat):
        """F_A of Sec. 3.3 for fine operator A (sparse) and augmentation Uhat [n, k]."""
        AH = (self.I.T @ A @ self.I).toarray()
        if Uhat is None or Uhat.shape[1] == 0:
            return AH
        AU = A @ Uhat
        bH = self.I.T @ AU
        beta = Uhat.T @ AU
        return np.block([[AH, bH], [bH.T, beta]])

    def mass_blocks(self, Uhat):
        if Uhat is None or Uhat.shape[1] == 0:
            return self.B_H.copy()
        MU = self.M @ Uhat
        cH = self.I.T @ MU
        gamma = Uhat.T @ MU
        return np.block([[self.B_H, cH], [cH.T, gamma]])

    def eig_small(self, FA, FB):
        lam, U = sla.eigh(FA, FB, subset_by_index=[0, self.N - 1])
        return lam, U

    def basis_apply(self, Uhat, U):
        """Psi = I u_H + Uhat alpha for U = (u_H; alpha)."""
        nH = self.coarse.n
        Psi = self.I @ U[:nH]
        if Uhat is not None and Uhat.shape[1] > 0:
            Psi = Psi + Uhat @ U[nH:]
        return Psi

    # ------------------------------------------------------------ inner SCF
    def inner_scf(self, Uhat, rho_start, VH_start=None, tol=None, max_inner=None):
        inst = self.inst
        tol = inst.tol_scf if tol is None else tol
        max_inner = inst.max_inner if max_inner is None else max_inner
        FB = self.mass_blocks(Uhat)
        mixer = Anderson(self.fine.Wq, depth=getattr(inst, "anderson_depth", 5),
                         beta=getattr(inst, "anderson_beta", 0.7))
        rho_in = rho_start.copy()
        VH_prev = VH_start
        hist = []
        restart = float(getattr(inst, "anderson_restart", 0.0))
        for t in range(max_inner):
            VH, VHq, eps, vxc = self.nonlinear(rho_in, VH_prev)
            VH_prev = VH
            A = (self.AL + self.A_NL(VHq, vxc)).tocsr()
            FA = self.small_blocks(A, Uhat)
            lam, U = self.eig_small(FA, FB)
            occ, mts = self.occupations(lam)
            Psi = self.basis_apply(Uhat, U)
            rho_out = self.density(Psi, occ)
            res = self.norm0(rho_out - rho_in)
            hist.append(res)
            if res < tol:
                return State(lam, Psi, rho_in, rho_out, VH, occ, mts, t + 1, res, True,
                             {"res_hist": hist, "U": U, "eps": eps, "vxc": vxc, "VHq": VHq})
            if t == max_inner - 1:
                break
            # optional safeguard: a residual above `restart` x the best one of
            # this inner SCF clears the history (the next mix is linear)
            if restart > 0.0 and t > 0 and res > restart * min(hist[:-1]):
                mixer.hist.clear()
            rho_in = mixer.mix(rho_in, rho_out)
        return State(lam, Psi, rho_in, rho_out, VH, occ, mts, max_inner, res, False,
                     {"res_hist": hist, "U": U, "eps": eps, "vxc": vxc, "VHq": VHq})

    # ------------------------------------------------------------ Algorithm 3
    def initial_state(self):
        if self.coarse.n < self.N:
            raise ValueError("the coarse-space initial guess needs dim S_H >= N")
        zero = np.zeros_like(self.fine.Wq)
        return self.inner_scf(None, zero)

    def bvp(self, st):
        """Step 1 of Algorithm 3: the N shifted linear problems."""
        _, VHq, _, vxc = self.nonlinear_cached(st)
        Ht = (self.AL + self.A_NL(VHq, vxc) + self.mu * self.M).tocsr()
        R = (self.M @ st.Psi) * (st.lam + self.mu)[None, :]
        return solve_spd(Ht, R, tol=self.inst.tol_bvp * 1e-1)

    def nonlinear_cached(self, st):
        VHq = self.fine.at_quad(st.VH)
        if self.inst.xc:
            eps, vxc = lda.lda(st.rho_in)
        else:
            eps = np.zeros_like(st.rho_in)
            vxc = np.zeros_like(st.rho_in)
        return st.VH, VHq, eps, vxc

    def augment_basis(self, Uhat):
        """M-orthonormal basis of the M-orthogonal complement of span{Uhat} to I S_H."""
        c = self.I.T @ (self.M @ Uhat)
        Y = sla.cho_solve(self.B_H_chol, c)
        U = Uhat - self.I @ Y
        g = U.T @ (self.M @ U)
        L = np.linalg.cholesky(0.5 * (g + g.T))
        return sla.solve_triangular(L, U.T, lower=True).T

    def step(self, st):
        Uhat = self.augment_basis(self.bvp(st))
        new = self.inner_scf(Uhat, st.rho_in, VH_start=st.VH)
        new.info["Uhat"] = Uhat
        new.info["drho"] = self.norm0(new.rho_out - st.rho_out)
        return new

    def solve(self, st=None, max_outer=None, tol=None, callback=None):
        st = self.initial_state() if st is None else st
        max_outer = self.inst.max_outer if max_outer is None else max_outer
        tol = self.inst.tol_scf if tol is None else tol
        for l in range(max_outer):
            st = self.step(st)
            if callback is not None:
                callback(l, st)
            if st.info["drho"] < tol:
                break
        return st

    # ------------------------------------------------------------ energies
    def energy(self, st):
        """Sec. 3.1 energy formula at the density rho_in of the potential."""
        f = self.fine
        _, VHq, eps, vxc = self.nonlinear_cached(st)
        rho = st.rho_in
        occ = self.occ if st.occ is None else st.occ
        return (float(np.dot(occ, st.lam))
                - f.integrate((0.5 * VHq + vxc) * rho)
                + f.integrate(rho * eps) + self.Enn + st.minus_TS)

    def energy_gradient(self, rho_q):
        """Hellmann-Feynman gradient of the total energy with respect to the
        nuclear positions and charges on a fixed mesh: int rho dV_ext/dp plus
        d E_nn/dp, [M, 4] (x, y, z, Z).  Exact for the discrete variational
        problem at self-consistency (the basis does not move with the nuclei)."""
        dV = dvext_dparams(self.inst, self.fine.xq)
        g = np.einsum("eq,kceq->kc", self.fine.Wq * rho_q, dV)
        return g + nuclear_repulsion_grad(self.inst)

    def bvp_vjp(self, st, Uhat, G):
        """Vector-Jacobian product of the linear problems H~ U^ = R (R fixed)
        with respect to the nuclear parameters: for L with dL/dU^ = G, the
        adjoint A = H~^-1 G (H~ symmetric) gives dL/dp = -sum_q W_q dV/dp
        sum_c a_c(x_q) u_c(x_q), [M, 4]."""
        _, VHq, _, vxc = self.nonlinear_cached(st)
        Ht = (self.AL + self.A_NL(VHq, vxc) + self.mu * self.M).tocsr()
        A = solve_spd(Ht, G, tol=1e-15)
        f = self.fine
        aq = f.at_quad(f.to_nodes(A))
        uq = f.at_quad(f.to_nodes(Uhat))
        prod = np.einsum("eqc,eqc->eq", aq, uq)
        dV = dvext_dparams(self.inst, f.xq)
        return -np.einsum("eq,kceq->kc", f.Wq * prod, dV)

    def variational_energy(self, Psi):
        """E(Psi) of Sec. 2 (kinetic + external + xc + Hartree/2 + E_nn)."""
        f = self.fine
        rho = self.density(Psi)
        kin = 0.5 * float(np.sum(self.occ * np.einsum("in,in->n", Psi, self.K @ Psi)))
        ext = f.integrate(self.vext_q * rho)
        E = kin + ext + self.Enn
        if self.inst.xc:
            eps, _ = lda.lda(rho)
            E += f.integrate(rho * eps)
        if self.inst.hartree:
            VH = hartree.hartree(f, self.K, self.K_IB, rho, tol=1e-14)
            E += 0.5 * f.integrate(f.at_quad(VH) * rho)
        return E

    # ------------------------------------------------------------ direct SCF (plain definition)
    def direct_scf(self, tol=None, max_iter=200, dense_max=4000):
        """SCF on the whole fine space: the discrete ground state of Sec. 2."""
        f = self.fine
        tol = self.inst.tol_scf if tol is None else tol
        Md = self.M.toarray() if f.n <= dense_max else None
        mixer = Anderson(f.Wq, depth=getattr(self.inst, "anderson_depth", 5),
                         beta=getattr(self.inst, "anderson_beta", 0.7))
        rho_in = np.zeros_like(f.Wq)
        VH_prev = None
        for t in range(max_iter):
            VH, VHq, eps, vxc = self.nonlinear(rho_in, VH_prev)
            VH_prev = VH
            A = (self.AL + self.A_NL(VHq, vxc)).tocsr()
            if Md is not None:
                lam, Psi = sla.eigh(A.toarray(), Md, subset_by_index=[0, self.N - 1])
            else:
                import scipy.sparse.linalg as spla
                lam, Psi = spla.eigsh(A, k=self.N, M=self.M, sigma=-1e3, which="LM", tol=1e-14)
                o = np.argsort(lam)
                lam, Psi = lam[o], Psi[:, o]
            occ, mts = self.occupations(lam)
            rho_out = self.density(Psi, occ)
            res = self.norm0(rho_out - rho_in)
            if res < tol:
                return State(lam, Psi, rho_in, rho_out, VH, occ, mts, t + 1, res, True)
            rho_in = mixer.mix(rho_in, rho_out)
        return State(lam, Psi, rho_in, rho_out, VH, occ, mts, max_iter, res, False)
