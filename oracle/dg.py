"""Acoustic / elastic nodal-DG right-hand side and AB3 stepping (oracle).

Test infrastructure: float64, numpy, one plain pass per operation.

Physics and penalty terms follow Section 2.1:
  acoustic  p_t + rho c^2 div v = 0,  rho v_t + grad p = 0,
            p_p = -(rho c^2)^- k_c a_c,  p_v = c^- k_c a_c,
            a_c = [[p]] - (rho c)^+ [[v_n]],  k_c = 1/{rho c},
            [[a]] = (a^+ - a^-)/2 (semi-jump), {a} = (a^- + a^+)/2;
  elastic   sigma_t = lambda (div v) I + 2 mu sym(grad v),  rho v_t = div sigma,
            P_sigma = k_p a_p lambda^- I + 2 (k_p a_p - k_s a_s) mu^- n(x)n
                      + 2 k_s mu^- sym(n (x) a_s_vec),
            p_v = (k_p a_p c_p^- - k_s a_s c_s^-) n + k_s c_s^- a_s_vec,
            a_p = [[s_nn]] + (rho c_p)^+ [[v_n]],  a_s = [[s_nn]] + (rho c_s)^+ [[v_n]],
            a_s_vec = [[sigma n]] + (rho c_s)^+ [[v]],  k_{p,s} = 1/{rho c_{p,s}}.
The variational forms of Section 2.1 put -int p_p psi, -int p_v n psi
(acoustic) and +int P_sigma psi, +int p_v psi (elastic) on the boundary.
The element RHS is Eq. dgLocalRhs:
  r_k = sum_ij g^vol_{k,i,j} D_j f_{j,k} + sum_f g^sur_{k,f} L_f p_{k,f},
evaluated here with the chain rule d/dx_i = sum_j g_{ij} D_j and
g^sur = Fscale.  Time stepping is Eq. updateScheme (AB3, a = (23,-16,5)/12).

Readings where the paper is silent (see the design notes):
* outer boundary: mirror ghost states.  Acoustic rigid wall:
  p+ = p-, v+ = v- - 2 (v-.n) n.  Elastic free surface (default):
  v+ = v-, sigma+ = -sigma-; elastic rigid: v+ = -v-, sigma+ = sigma-.
  Ghost coefficients equal the interior ones.
* centred flux (energy test): a* = {a} for every trace, i.e.
  acoustic dp = -kappa^- [[v_n]], dv = -(1/rho^-) [[p]] n; elastic
  dsigma = C^-: sym(n (x) [[v]]), dv = [[sigma n]] / rho^-.
* time step: dt = cfl / max(c Fscale ((N+1)(N+2)/2 + 2)), cfl = 0.4.
* AB3 start-up: Euler, then AB2 (3/2, -1/2), then AB3, unless a history
  r^{-1}, r^{-2} is supplied.
* point sources: amp(t_m) M_k^{-1} l(x_s) is added to r_p (acoustic) or
  amp(t_m) (d_i / rho_k) M_k^{-1} l(x_s) to r_{v_i} (elastic), in the tet
  whose smallest barycentric of x_s is largest; several sources add their
  terms.
"""

import numpy as np

from .refelem import RefElement
from .mesh import Mesh

ACOUSTIC, ELASTIC = "acoustic", "elastic"
AB3 = np.array([23.0, -16.0, 5.0]) / 12.0
AB2 = np.array([1.5, -0.5, 0.0])
EULER = np.array([1.0, 0.0, 0.0])
# elastic field order and the stress index map
ELASTIC_FIELDS = ("vx", "vy", "vz", "sxx", "syy", "szz", "sxy", "sxz", "syz")
SIG = np.array([[3, 6, 7], [6, 4, 8], [7, 8, 5]])


def nfields(model):
    return 4 if model == ACOUSTIC else 9


def acoustic_penalty(pM, pP, vM, vP, n, kappaM, rhoM, cM, ZP, flux="upwind"):
    """Penalty corrections (dp, dv) at face nodes, Section 2.1.

    Returns dp = -p_p and dv = -p_v n, the quantities that the strong-form
    RHS lifts: r_p += LIFT(Fscale dp), r_v += LIFT(Fscale dv).
    Upwind: a_c = [[p]] - Z^+ [[v_n]], k_c = 1/{Z}, dp = kappa^- k_c a_c,
    dv = -c^- k_c a_c n.  Centred: dp = -kappa^- [[v_n]], dv = -[[p]] n / rho^-.
    Shapes: p* [...], v* / n [..., 3], coefficients broadcastable to [...].
    """
    jp = 0.5 * (pP - pM)
    jvn = 0.5 * np.sum((vP - vM) * n, axis=-1)
    if flux == "upwind":
        ZM = rhoM * cM
        kc = 2.0 / (ZM + ZP)
        ac = jp - ZP * jvn
        dp = kappaM * kc * ac
        dv = -(cM * kc * ac)[..., None] * n
    else:
        dp = -kappaM * jvn
        dv = -(jp / rhoM)[..., None] * n
    return dp, dv


def elastic_penalty(vM, vP, sM, sP, n, lamM, muM, rhoM, ZpP, ZsP, flux="upwind"):
    """Penalty terms (P_sigma [..., 3, 3], p_v [..., 3]) of Section 2.1.

    Both are added (r += LIFT(Fscale P)).  Upwind (exact Riemann solver,
    Wilcox 2010):
      P_sigma = k_p a_p lam^- I + 2 (k_p a_p - k_s a_s) mu^- n(x)n + 2 k_s mu^- sym(n(x)a_s_vec)
      p_v     = (k_p a_p c_p^- - k_s a_s c_s^-) n + k_s c_s^- a_s_vec
    Centred: P_sigma = lam^- (n.[[v]]) I + 2 mu^- sym(n(x)[[v]]), p_v = [[sigma n]] / rho^-.
    Shapes: v* / n [..., 3], s* [..., 3, 3], coefficients broadcastable to [...].
    """
    n = np.broadcast_to(n, vM.shape)
    jv = 0.5 * (vP - vM)
    jsn = 0.5 * np.einsum("...ij,...j->...i", sP - sM, n)
    jvn = np.sum(jv * n, axis=-1)
    eye = np.eye(3)

    def sym_n(a):
        t = n[..., :, None] * a[..., None, :]
        return 0.5 * (t + np.swapaxes(t, -1, -2))

    if flux == "upwind":
        cpM = np.sqrt((lamM + 2 * muM) / rhoM)
        csM = np.sqrt(muM / rhoM)
        ZpM, ZsM = rhoM * cpM, rhoM * csM
        jsnn = np.sum(jsn * n, axis=-1)
        ap = jsnn + ZpP * jvn
        as_ = jsnn + ZsP * jvn
        asv = jsn + ZsP[..., None] * jv
        kp = 2.0 / (ZpM + ZpP)
        ks = 2.0 / (ZsM + ZsP)
        NN = n[..., :, None] * n[..., None, :]
        Psig = ((kp * ap * lamM)[..., None, None] * eye
                + (2.0 * (kp * ap - ks * as_) * muM)[..., None, None] * NN
                + (2.0 * ks * muM)[..., None, None] * sym_n(asv))
        pv = (kp * ap * cpM - ks * as_ * csM)[..., None] * n + (ks * csM)[..., None] * asv
    else:
        Psig = (lamM * jvn)[..., None, None] * eye + (2.0 * muM)[..., None, None] * sym_n(jv)
        pv = jsn / rhoM[..., None]
    return Psig, pv


class Solver:
    """Plain FP64 DG discretisation of one mesh."""

    def __init__(self, model, N, verts, tets, coeffs, flux="upwind", bc=None,
                 ref=None):
        self.model = model
        self.N = N
        self.ref = ref if ref is not None else RefElement(N)
        self.mesh = Mesh(self.ref, verts, tets)
        self.flux = flux
        self.bc = bc if bc is not None else ("rigid" if model == ACOUSTIC else "free")
        coeffs = np.asarray(coeffs, dtype=np.float64)
        K = self.mesh.K
        if model == ACOUSTIC:
            rho, c = coeffs[:, 0], coeffs[:, 1]
            self.rho, self.c = rho, c
            self.kappa = rho * c * c
            self.Z = rho * c
            self.cmax = c
        else:
            lam, mu, rho = coeffs[:, 0], coeffs[:, 1], coeffs[:, 2]
            self.lam, self.mu, self.rho = lam, mu, rho
            self.cp = np.sqrt((lam + 2 * mu) / rho)
            self.cs = np.sqrt(mu / rho)
            self.Zp, self.Zs = rho * self.cp, rho * self.cs
            self.cmax = self.cp
        self.Nf = nfields(model)
        self.K = K
        self.srcs = []  # (element, M_k^{-1} l(x_s), amplitudes, direction) per source

    # ------------------------------------------------------------------
    def node_coords(self):
        return self.mesh.x

    def suggest_dt(self, cfl=0.4):
        """dt = cfl * min_{k,f} 1 / (c_max,k Fscale_{k,f} ((N+1)(N+2)/2 + 2)).

        The degree factor follows the measured spectral radius of the upwind
        RHS operator (within ~10 % for N = 1..8); cfl = 0.4 keeps |lambda| dt
        <= 0.45, inside the AB3 stability region."""
        m = self.mesh
        nf = (self.N + 1) * (self.N + 2) / 2.0 + 2.0
        return cfl * float(np.min(1.0 / (self.cmax[:, None] * m.Fscale * nf)))

    # ------------------------------------------------------------------
    # E selects the elements whose RHS is computed (all of them when E is a
    # full slice); the traces still read the neighbours' states from q.
    def _traces(self, q, E):
        """Interior (-) and exterior (+) traces, [len(E), Nf, 4, Nfp] each."""
        m = self.mesh
        qf = q.transpose(1, 0, 2).reshape(self.Nf, -1)
        return qf[:, m.vmapM[E]].transpose(1, 0, 2, 3), qf[:, m.vmapP[E]].transpose(1, 0, 2, 3)

    def _lift(self, corr, E):
        """sum_f Fscale_f L_f corr_f for corr [len(E), Nf, 4, Nfp]."""
        m = self.mesh
        c = corr * m.Fscale[E][:, None, :, None]
        K = c.shape[0]
        return np.einsum("ij,kfj->kfi", self.ref.LIFT, c.reshape(K, self.Nf, -1))

    def _ref_grad(self, u):
        """[K, F, 3, Np]: (D_r u, D_s u, D_t u) for u [K, F, Np]."""
        R = self.ref
        return np.stack([np.einsum("ij,kfj->kfi", D, u) for D in (R.Dr, R.Ds, R.Dt)], axis=2)

    def _phys_grad(self, u, E=slice(None)):
        """[K, F, 3(i), Np]: d u / d x_i = sum_j g_ij D_j u (u of the elements E)."""
        return np.einsum("kij,kfjn->kfin", self.mesh.g[E], self._ref_grad(u))

    # ------------------------------------------------------------------
    def rhs(self, q, step=None, elems=None):
        """The semi-discrete RHS (Eq. dgLocalRhs) for the full state q; of
        every element, or only of the elements listed in elems (sampled
        checks of large meshes: the same formulas on those elements' rows)."""
        q = np.asarray(q, dtype=np.float64)
        E = slice(None) if elems is None else np.asarray(elems, dtype=np.int64)
        r = self._rhs_acoustic(q, E) if self.model == ACOUSTIC else self._rhs_elastic(q, E)
        for k, b, amp, d in (self.srcs if step is not None else []):
            a = amp[step] if step < len(amp) else 0.0
            rows = [k] if elems is None else list(np.nonzero(np.asarray(elems) == k)[0])
            for row in rows:
                if self.model == ACOUSTIC:
                    r[row, 0] += a * b
                else:
                    for i in range(3):
                        r[row, i] += a * d[i] / self.rho[k] * b
        return r

    def _rhs_acoustic(self, q, E):
        m = self.mesh
        qE = q[E]
        K = qE.shape[0]
        kappa, rho, c, Z = self.kappa[E], self.rho[E], self.c[E], self.Z[E]
        p, v = qE[:, 0:1], qE[:, 1:4]
        gp = self._phys_grad(p, E)[:, 0]                # [K, 3, Np]
        gv = self._phys_grad(v, E)                      # [K, 3(comp), 3(dir), Np]
        divv = np.einsum("kiin->kn", gv)
        r = np.empty_like(qE)
        r[:, 0] = -kappa[:, None] * divv
        r[:, 1:4] = -(1.0 / rho)[:, None, None] * gp

        qM, qP = self._traces(q, E)
        n = m.n[E][:, :, None, :]                       # [K, 4, 1, 3]
        pM, pP = qM[:, 0], qP[:, 0]
        vM = np.moveaxis(qM[:, 1:4], 1, -1)             # [K, 4, Nfp, 3]
        vP = np.moveaxis(qP[:, 1:4], 1, -1)
        bnd = m.boundary[E][:, :, None]
        vnM = np.sum(vM * n, axis=-1)
        # rigid-wall mirror ghost
        pP = np.where(bnd, pM, pP)
        vP = np.where(bnd[..., None], vM - 2.0 * vnM[..., None] * n, vP)
        ZP = np.where(bnd, Z[:, None, None], self.Z[m.EToE[E]][:, :, None])
        dp, dv = acoustic_penalty(pM, pP, vM, vP, n, kappa[:, None, None],
                                  rho[:, None, None], c[:, None, None], ZP,
                                  self.flux)
        corr = np.empty((K, 4, 4, self.ref.Nfp))
        corr[:, 0] = dp
        corr[:, 1:4] = np.moveaxis(dv, -1, 1)
        return r + self._lift(corr, E)

    def _rhs_elastic(self, q, E):
        m = self.mesh
        qE = q[E]
        K = qE.shape[0]
        lam, mu, rho = self.lam[E], self.mu[E], self.rho[E]
        v = qE[:, 0:3]
        gv = self._phys_grad(v, E)                       # [K, i(comp), j(dir), Np]
        divv = np.einsum("kiin->kn", gv)
        r = np.empty_like(qE)
        for i in range(3):
            for j in range(i, 3):
                val = mu[:, None] * (gv[:, i, j] + gv[:, j, i])
                if i == j:
                    val = val + lam[:, None] * divv
                r[:, SIG[i, j]] = val
        sig = qE[:, SIG.ravel()].reshape(K, 3, 3, -1)     # sigma_ij
        gs = self._phys_grad(sig.reshape(K, 9, -1), E).reshape(K, 3, 3, 3, -1)  # d_k sigma_ij
        divs = np.einsum("kijjn->kin", gs)
        r[:, 0:3] = divs / rho[:, None, None]

        qM, qP = self._traces(q, E)
        n = m.n[E][:, :, None, :]                        # [K, 4, 1, 3]
        vM = np.moveaxis(qM[:, 0:3], 1, -1)              # [K, 4, Nfp, 3]
        vP = np.moveaxis(qP[:, 0:3], 1, -1)
        sM = np.moveaxis(qM[:, SIG.ravel()], 1, -1).reshape(qM.shape[0], 4, -1, 3, 3)
        sP = np.moveaxis(qP[:, SIG.ravel()], 1, -1).reshape(qP.shape[0], 4, -1, 3, 3)
        bnd = m.boundary[E][:, :, None]
        if self.bc == "free":
            vP = np.where(bnd[..., None], vM, vP)
            sP = np.where(bnd[..., None, None], -sM, sP)
        else:
            vP = np.where(bnd[..., None], -vM, vP)
            sP = np.where(bnd[..., None, None], sM, sP)
        def nb(x):
            return np.where(bnd, x[E][:, None, None], x[m.EToE[E]][:, :, None])
        Psig, pv = elastic_penalty(vM, vP, sM, sP, n, lam[:, None, None], mu[:, None, None],
                                   rho[:, None, None], nb(self.Zp), nb(self.Zs), self.flux)
        corr = np.empty((K, 9, 4, self.ref.Nfp))
        corr[:, 0:3] = np.moveaxis(pv, -1, 1)
        for i in range(3):
            for j in range(i, 3):
                corr[:, SIG[i, j]] = Psig[..., i, j]
        return r + self._lift(corr, E)

    # ------------------------------------------------------------------
    def locate(self, xs):
        """Element whose smallest barycentric coordinate of xs is largest, and
        the reference coordinates of xs in it (affine map of Section 2.2)."""
        m = self.mesh
        xs = np.asarray(xs, dtype=np.float64)
        x1 = m.verts[m.tets[:, 0]]
        rst = np.einsum("kij,kj->ki", np.linalg.inv(m.A), xs[None, :] - x1) - 1.0
        lam = np.stack([-(1 + rst.sum(axis=1)) / 2.0, (1 + rst[:, 0]) / 2.0,
                        (1 + rst[:, 1]) / 2.0, (1 + rst[:, 2]) / 2.0], axis=1)
        k = int(np.argmax(lam.min(axis=1)))
        return k, rst[k]

    def point_values(self, q, pts):
        """[npts, Nf]: the nodal polynomial of the containing element evaluated
        at each point, sum_i q_k[f][i] l_i(r(x)) (Section 2.2)."""
        out = np.empty((len(pts), self.Nf))
        for p, x in enumerate(pts):
            k, rst = self.locate(x)
            ell = self.ref.lag.eval(rst[None, :])[0]
            out[p] = np.asarray(q[k], dtype=np.float64) @ ell
        return out

    def set_source(self, xs, amp, direction=(0.0, 0.0, 1.0)):
        """One point source at xs (replacing any others); returns its tet."""
        self.srcs = []
        return self.add_source(xs, amp, direction)

    def add_source(self, xs, amp, direction=(0.0, 0.0, 1.0)):
        """One more point source at xs; returns its tet."""
        m, R = self.mesh, self.ref
        xs = np.asarray(xs, dtype=np.float64)
        x1 = m.verts[m.tets[:, 0]]
        rst = np.einsum("kij,kj->ki", np.linalg.inv(m.A), xs[None, :] - x1) - 1.0
        lam = np.stack([-(1 + rst.sum(axis=1)) / 2.0, (1 + rst[:, 0]) / 2.0,
                        (1 + rst[:, 1]) / 2.0, (1 + rst[:, 2]) / 2.0], axis=1)
        k = int(np.argmax(lam.min(axis=1)))
        ell = R.lag.eval(rst[k][None, :])[0]
        b = R.Minv @ ell / m.J[k]
        self.srcs.append((k, b, np.asarray(amp, dtype=np.float64), np.asarray(direction, dtype=np.float64)))
        return k

    # ------------------------------------------------------------------
    def energy(self, q):
        m, M = self.mesh, self.ref.M

        def ip(a, b):  # per element int a b  (reference measure)
            return np.einsum("ki,ij,kj->k", a, M, b)

        if self.model == ACOUSTIC:
            e = ip(q[:, 0], q[:, 0]) / self.kappa
            for i in range(1, 4):
                e = e + self.rho * ip(q[:, i], q[:, i])
        else:
            lam, mu = self.lam, self.mu
            e = sum(self.rho * ip(q[:, i], q[:, i]) for i in range(3))
            ss = sum(ip(q[:, 3 + i], q[:, 3 + i]) for i in range(3)) + \
                2.0 * sum(ip(q[:, 6 + i], q[:, 6 + i]) for i in range(3))
            tr = q[:, 3] + q[:, 4] + q[:, 5]
            e = e + (ss - lam / (3 * lam + 2 * mu) * ip(tr, tr)) / (2 * mu)
        return 0.5 * float(np.sum(m.J * e))

    def energy_rate(self, q, r):
        """d/dt E_h along the semi-discrete flow: the bilinear form of energy(q) with r."""
        m, M = self.mesh, self.ref.M

        def ip(a, b):
            return np.einsum("ki,ij,kj->k", a, M, b)

        if self.model == ACOUSTIC:
            e = ip(q[:, 0], r[:, 0]) / self.kappa
            for i in range(1, 4):
                e = e + self.rho * ip(q[:, i], r[:, i])
        else:
            lam, mu = self.lam, self.mu
            e = sum(self.rho * ip(q[:, i], r[:, i]) for i in range(3))
            ss = sum(ip(q[:, 3 + i], r[:, 3 + i]) for i in range(3)) + \
                2.0 * sum(ip(q[:, 6 + i], r[:, 6 + i]) for i in range(3))
            trq = q[:, 3] + q[:, 4] + q[:, 5]
            trr = r[:, 3] + r[:, 4] + r[:, 5]
            e = e + (ss - lam / (3 * lam + 2 * mu) * ip(trq, trr)) / (2 * mu)
        return float(np.sum(m.J * e))


class AB3Stepper:
    """q^{m+1} = q^m + dt sum_s a_s r^{m-s+1} (Eq. updateScheme)."""

    def __init__(self, solver, q0, dt, history=None, t0=0.0):
        self.s = solver
        self.q = np.array(q0, dtype=np.float64)
        self.dt = float(dt)
        self.m = 0
        self.t0 = t0
        if history is None:
            self.r1 = np.zeros_like(self.q)
            self.r2 = np.zeros_like(self.q)
            self.have = 0
        else:
            self.r1, self.r2 = (np.array(h, dtype=np.float64) for h in history)
            self.have = 2

    def step(self, n=1):
        for _ in range(n):
            r = self.s.rhs(self.q, step=self.m)
            a = AB3 if self.have >= 2 else (AB2 if self.have == 1 else EULER)
            self.q = self.q + self.dt * (a[0] * r + a[1] * self.r1 + a[2] * self.r2)
            self.r2, self.r1 = self.r1, r
            self.have = min(self.have + 1, 2)
            self.m += 1
        return self.q
