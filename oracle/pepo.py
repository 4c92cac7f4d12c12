"""The operator network and the literal bond update (oracle, complex128).

State (Sec. 2.3 "Pauli Basis Tensor Network", Sec. 3.1 IsingState):
  O[v]      site tensor with axes [legs in canonical order ..., s, s'].  The
            physical pair is a literal 2x2 operator block (the GPU path uses
            the 4 real Pauli coefficients instead; the two differ by a fixed
            change of basis on the physical leg).
  M[(u,v)]  double-layer message from u into v: the environment of v's leg
            toward u.  Convention: M[j, j'] pairs conj(O_v) at index j with
            O_v at index j'.
  lam[b]    Vidal-normalised singular values of bond b (Eq. 12).

Initial state (Sec. 2.3, Fig. 1): the observable Pauli at site c, the identity
elsewhere, every bond dimension 1 and every message [[1]].

Bond update (Sec. 2.5, Eqs. 11-12).  The update of the pair (v1, v2) is a
gauge change, a reduction, the gate, a truncation and the inverse gauge
change, in that order because each step needs the one before it:
  * Gauge.  The converged double-layer messages are Gram matrices of the
    environment seen by each leg; their (pseudo) square roots, from the
    eigen-decomposition of the Hermitian part with eigenvalues below
    pinv_rel times the largest set to zero, are absorbed on every leg but
    the shared bond, so the bond sees an orthonormalised environment.
  * Reduction.  Each site, reshaped to (environment legs) x (bond, s, s'),
    factors as Q R (numpy's Householder QR); the isometry Q does not take
    part in the gate, so only the two small R factors are contracted over
    the bond into the two-site block.
  * Gate.  The two-site Heisenberg-picture conjugation g^dagger (.) g acts
    on the two physical pairs of the block.
  * Truncation (Eq. 11).  The SVD of the block keeps
    chi_new = min(#{s_i >= eps_cut s_0}, chi_max) values; U sqrt(S) and
    sqrt(S) V^H (raw singular values) become the new R factors.
  * Inverse gauge.  The new R factors are multiplied back into Q, the legs
    return to canonical order, the absorbed square roots are removed with
    the pseudo-inverse square roots, and the bond's messages become
    diag(lam) with lam = s / ||s_kept|| (Eq. 12).

Pinned by: tests/test_oracle_pepo.py -- without truncation the network
contracts to the dense operator exactly on a 3 x 3 grid (loops) and on chains;
on chains the gate-time lam equal the dense operator-Schmidt values; the
closed forms at J = 0 / h = 0 hold through the whole pipeline.
"""
import numpy as np

from . import gates as G
from .lattice import legs_of, site_index


def bond_key(a, b):
    return (a, b) if a < b else (b, a)


def leg_apply(T, k, S):
    """out[..., i, ...] = sum_j S[i, j] T[..., j, ...] on axis k."""
    return np.moveaxis(np.tensordot(S, T, axes=([1], [k])), 0, k)


def env_sqrt(M, pinv_rel):
    """Pseudo square root and pseudo inverse square root of a PSD message."""
    Ms = 0.5 * (M + M.conj().T)
    w, V = np.linalg.eigh(Ms)
    wmax = max(float(np.max(w)), 0.0)
    keep = w > pinv_rel * wmax
    wk = np.where(keep, w, 1.0)
    sq = np.where(keep, np.sqrt(wk), 0.0)
    isq = np.where(keep, 1.0 / np.sqrt(wk), 0.0)
    S = (V * sq) @ V.conj().T
    Si = (V * isq) @ V.conj().T
    return S, Si


class Network:
    def __init__(self, Lx, Ly, obs_xy, obs_pauli="Z"):
        if Lx * Ly < 2:
            raise ValueError("the method needs at least two sites")
        self.Lx, self.Ly = Lx, Ly
        self.N = Lx * Ly
        self.obs_site = site_index(obs_xy[0], obs_xy[1], Lx)
        self.obs_pauli = obs_pauli
        self.legs = []
        self.O = []
        for v in range(self.N):
            x, y = v % Lx, v // Lx
            lg = legs_of(x, y, Lx, Ly)
            self.legs.append(lg)
            P = G.PAULI[obs_pauli] if v == self.obs_site else G.I2
            self.O.append(P.reshape((1,) * len(lg) + (2, 2)).astype(np.complex128))
        self.M = {}
        self.lam = {}
        for v in range(self.N):
            for (_, u) in self.legs[v]:
                self.M[(u, v)] = np.ones((1, 1), dtype=np.complex128)
                self.lam[bond_key(u, v)] = np.ones(1)

    def axis(self, v, u):
        for k, (_, w) in enumerate(self.legs[v]):
            if w == u:
                return k
        raise KeyError((v, u))

    def chi(self, a, b):
        return self.O[a].shape[self.axis(a, b)]

    def copy(self):
        n = Network.__new__(Network)
        n.__dict__.update(self.__dict__)
        n.O = [o.copy() for o in self.O]
        n.M = {k: m.copy() for k, m in self.M.items()}
        n.lam = {k: l.copy() for k, l in self.lam.items()}
        n.legs = [list(l) for l in self.legs]
        return n


def from_pauli(Lx, Ly, obs_xy, obs_pauli, sites, chi, msgs, sites_subset=None):
    """Network from Pauli-basis arrays (canonical [U, D, L, R, p] layout).

    O_v = sum_p psi_v[..., p] P_p (Sec. 2.3: psi holds Pauli coefficients).
    chi / msgs are indexed by the library's bond numbering (horizontal bonds
    first); msgs[b, 0] is the message first site -> second site.  With
    sites_subset only those site tensors are converted (others left None).
    """
    net = Network(Lx, Ly, obs_xy, obs_pauli)
    P = np.stack(G.PAULI_BY_INDEX)
    bid = {}
    for y in range(Ly):
        for x in range(Lx - 1):
            bid[(y * Lx + x, y * Lx + x + 1)] = y * (Lx - 1) + x
    for y in range(Ly - 1):
        for x in range(Lx):
            bid[(y * Lx + x, (y + 1) * Lx + x)] = Ly * (Lx - 1) + y * Lx + x
    for v in range(net.N):
        if sites_subset is not None and v not in sites_subset:
            net.O[v] = None
            continue
        psi = np.asarray(sites[v], dtype=np.float64)
        net.O[v] = np.tensordot(psi, P, axes=([psi.ndim - 1], [0])).astype(np.complex128)
    for (a, b), k in bid.items():
        c = int(chi[k])
        net.M[(a, b)] = np.asarray(msgs[k][0][:c, :c], dtype=np.complex128)
        net.M[(b, a)] = np.asarray(msgs[k][1][:c, :c], dtype=np.complex128)
    return net


def apply_site_gate(net, v, g):
    """O_v -> g^dagger O_v g on one site."""
    net.O[v] = np.einsum("ab,...bc,cd->...ad", g.conj().T, net.O[v], g)


def apply_site_gates(net, g):
    """O_v -> g^dagger O_v g on every site (Fig. 1, apply_unary_gate)."""
    gd = g.conj().T
    for v in range(net.N):
        net.O[v] = np.einsum("ab,...bc,cd->...ad", gd, net.O[v], g)


def _absorbed_matrix(net, v, other, pinv_rel):
    """The gauged site: square-rooted messages on every leg but the cut, the
    cut moved next to the physical pair, as an (env) x (cut, s, s') matrix."""
    O = net.O[v]
    deg = len(net.legs[v])
    kc = net.axis(v, other)
    inv = {}
    cv = O
    for k, (_, u) in enumerate(net.legs[v]):
        if u == other:
            continue
        S, Si = env_sqrt(net.M[(u, v)], pinv_rel)
        cv = leg_apply(cv, k, S)
        inv[k] = Si
    perm = [k for k in range(deg) if k != kc] + [kc, deg, deg + 1]
    cvp = np.transpose(cv, perm)
    env_shape = cvp.shape[: deg - 1]
    chi_c = cvp.shape[deg - 1]
    m = int(np.prod(env_shape)) if deg > 1 else 1
    return cvp.reshape(m, chi_c * 4), env_shape, perm, inv


def bond_update(net, v1, v2, g, chi_max, eps_cut, pinv_rel):
    """Apply the two-site gate g (4x4, qubit order (v1, v2)) to bond (v1, v2)."""
    mat1, env1, perm1, inv1 = _absorbed_matrix(net, v1, v2, pinv_rel)
    mat2, env2, perm2, inv2 = _absorbed_matrix(net, v2, v1, pinv_rel)
    Q1, R1 = np.linalg.qr(mat1)
    Q2, R2 = np.linalg.qr(mat2)
    k1, k2 = R1.shape[0], R2.shape[0]
    chi_c = mat1.shape[1] // 4
    R1r = R1.reshape(k1, chi_c, 2, 2)
    R2r = R2.reshape(k2, chi_c, 2, 2)
    RR4 = np.einsum("acxy,bczw->axybzw", R1r, R2r)
    g4 = g.reshape(2, 2, 2, 2)
    Rt = np.einsum("ijkl,aimbjn,mnoq->akoblq", g4.conj(), RR4, g4)
    U, s, Vh = np.linalg.svd(Rt.reshape(k1 * 4, k2 * 4), full_matrices=False)
    s0 = s[0]
    if not s0 > 0:
        raise FloatingPointError("bond matrix vanished")
    nkeep = int(np.sum(s >= eps_cut * s0))
    chi_new = max(1, min(nkeep, chi_max))
    tot = float(np.sum(s ** 2))
    disc = float(np.sum(s[chi_new:] ** 2)) / tot
    sk = s[:chi_new]
    lam = sk / np.linalg.norm(sk)
    rs = np.sqrt(sk)
    M1 = (U[:, :chi_new] * rs).reshape(k1, 2, 2, chi_new).transpose(0, 3, 1, 2)
    M2 = (rs[:, None] * Vh[:chi_new]).reshape(chi_new, k2, 2, 2).transpose(1, 0, 2, 3)
    for (v, Q, Mi, env, perm, inv, k) in ((v1, Q1, M1, env1, perm1, inv1, k1),
                                           (v2, Q2, M2, env2, perm2, inv2, k2)):
        cvn = (Q @ Mi.reshape(k, chi_new * 4)).reshape(tuple(env) + (chi_new, 2, 2))
        On = np.transpose(cvn, np.argsort(perm))
        for kk, Si in inv.items():
            On = leg_apply(On, kk, Si)
        net.O[v] = On
    D = np.diag(lam).astype(np.complex128)
    net.M[(v1, v2)] = D.copy()
    net.M[(v2, v1)] = D.copy()
    net.lam[bond_key(v1, v2)] = lam
    return {"s": s, "lam": lam, "chi": chi_new, "disc": disc}
