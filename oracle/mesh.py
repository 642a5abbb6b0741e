"""Per-element geometry and connectivity (oracle; test infrastructure).

Section 2.2 leaves the geometric factors to the cited paper [Modave2015].
The readings used here, written from the affine map of a straight-sided
tetrahedron:

* x(r,s,t) = x1 + A (1+r, 1+s, 1+t), A = [x2-x1 | x3-x1 | x4-x1] / 2, J = det A;
* volume factor g^vol_{i,j} = d r_j / d x_i (entries of A^{-1}, transposed),
  as forced by the acoustic RHS of Section 3.2, where div v is written
  sum_i sum_j g_{ij} D_j v_i;
* for a face with reference normal N_f (area vector 2 N_f), the physical
  normal is n = g N_f / |g N_f| and the surface factor is
  g^sur = Fscale = sJ / J = |g N_f| (sJ = physical face area / 2);
* faces are matched by their sorted global vertex triples; face nodes by
  physical coordinates (nearest point).
"""

import numpy as np

from .refelem import FACE_VERTS, REF_NORMALS


class Mesh:
    def __init__(self, ref, verts, tets):
        self.ref = ref
        verts = np.asarray(verts, dtype=np.float64)
        tets = np.asarray(tets, dtype=np.int64)
        self.verts, self.tets = verts, tets
        K = tets.shape[0]
        self.K = K
        x1, x2, x3, x4 = (verts[tets[:, i]] for i in range(4))
        A = np.stack([x2 - x1, x3 - x1, x4 - x1], axis=2) / 2.0  # A[k, i, j] = dx_i/dr_j
        self.A = A
        self.J = np.linalg.det(A)
        if np.any(self.J <= 0):
            raise ValueError("non-positive Jacobian (inverted or degenerate tet)")
        Ainv = np.linalg.inv(A)
        self.g = np.transpose(Ainv, (0, 2, 1))  # g[k, i, j] = d r_j / d x_i
        nvec = np.einsum("kij,fj->kfi", self.g, REF_NORMALS)  # [K, 4, 3]
        self.Fscale = np.linalg.norm(nvec, axis=2)            # [K, 4]
        self.n = nvec / self.Fscale[:, :, None]
        self.sJ = self.Fscale * self.J[:, None]
        # physical node coordinates [K, Np, 3]
        rst1 = ref.nodes + 1.0
        self.x = x1[:, None, :] + np.einsum("kij,nj->kni", A, rst1)
        self._connect()

    def _connect(self):
        K, ref = self.K, self.ref
        Nfp, Np = ref.Nfp, ref.Np
        fv = np.stack([self.tets[:, list(FACE_VERTS[f])] for f in range(4)], axis=1)  # [K,4,3]
        keys = np.sort(fv.reshape(-1, 3), axis=1)
        order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
        sk = keys[order]
        same = np.all(sk[1:] == sk[:-1], axis=1)
        if np.any(same[1:] & same[:-1]):
            raise ValueError("non-conforming mesh: a face is shared by more than two tets")
        EToE = np.repeat(np.arange(K)[:, None], 4, axis=1)
        EToF = np.repeat(np.arange(4)[None, :], K, axis=0)
        i = np.nonzero(same)[0]
        a, b = order[i], order[i + 1]
        EToE.reshape(-1)[a] = b // 4
        EToF.reshape(-1)[a] = b % 4
        EToE.reshape(-1)[b] = a // 4
        EToF.reshape(-1)[b] = a % 4
        self.EToE, self.EToF = EToE, EToF
        self.boundary = (EToE == np.arange(K)[:, None]) & (EToF == np.arange(4)[None, :])

        # face-node matching by physical coordinates
        Fm = ref.Fmask
        own = np.arange(K)[:, None, None] * Np + Fm[None, :, :]          # [K,4,Nfp]
        vmapP = own.copy()
        h = np.cbrt(np.mean(self.J)) if K else 1.0
        tol = 1e-8 * h
        kk, ff = np.nonzero(~self.boundary)
        chunk = 20000
        for s in range(0, len(kk), chunk):
            k1, f1 = kk[s:s + chunk], ff[s:s + chunk]
            k2, f2 = EToE[k1, f1], EToF[k1, f1]
            xo = self.x[k1[:, None], Fm[f1]]                              # [c,Nfp,3]
            xn = self.x[k2[:, None], Fm[f2]]
            d = np.linalg.norm(xo[:, :, None, :] - xn[:, None, :, :], axis=3)
            j = np.argmin(d, axis=2)
            if np.max(np.take_along_axis(d, j[:, :, None], axis=2)) > tol:
                raise ValueError("face nodes of neighbouring tets do not coincide")
            vmapP[k1, f1] = k2[:, None] * Np + Fm[f2][np.arange(len(k2))[:, None], j]
        self.vmapM = own
        self.vmapP = vmapP
