"""The XY-model workload of the Supplemental Material, section "XY Model" (test infrastructure
only; see oracle/__init__.py).

Eq. XY_hamiltonian: H_XY = (g/2) sum_<ij> (X_i X_j + Y_i Y_j) on an Lx x Ly grid with open
boundaries, one qubit per MPS site.  Eq. xy_trotter_step: the depth-7 second-order product
  U(dt) = e^{-i dt H_A/2} e^{-i dt H_B/2} e^{-i dt H_C/2} e^{-i dt H_D} e^{-i dt H_C/2} e^{-i dt H_B/2}
          e^{-i dt H_A/2},
H_A / H_B the horizontal bonds starting on even / odd columns, H_C / H_D the vertical bonds
starting on even / odd rows (the bonds of one set do not overlap, so its gates commute).
Eq. xy_init: |psi_0(tau)> = exp(-i pi/8 H_Z) exp(-i tau H_XY) |Neel>, H_Z = sum_j (-1)^j Z_j,
|Neel> the ground state of H_Z; exp(-i tau H_XY) by Trotter steps of g dtau = 0.02 pi (1, 3 and 5
steps for g tau = 0.02 pi, 0.06 pi, 0.10 pi).  Eq. xy_signal: X^2(t) = (1/n^2) sum_{j,k}
(-1)^{j-k} <X_j X_k>.  The quench runs at g dt = 0.05 pi.

Readings where the section is silent:
* qubit (r, c) has index j = r Ly + c; the staggered sign (-1)^j is the checkerboard
  (-1)^{r + c} (the Neel pattern of the square lattice; for even Ly the parity of r Ly + c would
  give stripes);
* |Neel>: Z_j = -(-1)^j, i.e. qubit j is |1> where (-1)^{r+c} = +1 and |0> elsewhere;
* one qubit per MPS site along the row snake: row r runs c = 0 .. Ly-1 for even r and backwards
  for odd r;
* each two-qubit factor exp(-i s (g/2)(X X + Y Y)) of a layer of duration s is applied as one
  gate; non-adjacent sites are brought together by SWAP routing (oracle.mps, route "swap"), the
  only route of this workload; the gates of one layer are applied in the order of their
  (first site, second site) positions.
"""
import numpy as np

from . import mps
from . import statevector as sv

G_PAPER = 1.0
DT_PAPER = 0.05 * np.pi
DTAU_PAPER = 0.02 * np.pi
PREP_STEPS = {"low": 1, "mid": 3, "high": 5}  # g tau = 0.02 pi, 0.06 pi, 0.10 pi
LAYERS = (("A", 0.5), ("B", 0.5), ("C", 0.5), ("D", 1.0), ("C", 0.5), ("B", 0.5), ("A", 0.5))


def qid(Ly, r, c):
    return r * Ly + c


def stag_sign(Ly, j):
    """(-1)^j read as the checkerboard (-1)^{r + c}."""
    r, c = divmod(j, Ly)
    return 1 - 2 * ((r + c) & 1)


def bonds(Lx, Ly):
    """Nearest-neighbour pairs (j, k), j < k, of the open grid with their set A, B, C or D."""
    out = []
    for r in range(Lx):
        for c in range(Ly):
            if c + 1 < Ly:
                out.append((qid(Ly, r, c), qid(Ly, r, c + 1), "A" if c % 2 == 0 else "B"))
            if r + 1 < Lx:
                out.append((qid(Ly, r, c), qid(Ly, r + 1, c), "C" if r % 2 == 0 else "D"))
    return out


def blocks(Lx, Ly):
    """Sites of the one-to-one row snake in MPS order: dicts {qubits, d = 2}."""
    out = []
    for r in range(Lx):
        for i in range(Ly):
            c = i if r % 2 == 0 else Ly - 1 - i
            out.append({"row": r, "qubits": [qid(Ly, r, c)], "d": 2})
    return out


def schedule(Lx, Ly):
    """{set: [(p, q, j, k, 0, 0), ...]} with p < q the MPS positions of the pair, sorted."""
    pos = {b["qubits"][0]: p for p, b in enumerate(blocks(Lx, Ly))}
    out = {s: [] for s in "ABCD"}
    for (j, k, s) in bonds(Lx, Ly):
        p, q = pos[j], pos[k]
        out[s].append((p, q, j, k, 0, 0) if p < q else (q, p, k, j, 0, 0))
    for s in out:
        out[s].sort(key=lambda g: (g[0], g[1], g[2], g[3]))
    return out


def gate(theta):
    """exp(-i theta (X X + Y Y)) in the basis |q_a q_b> (first qubit most significant):
    X X + Y Y maps |01> <-> 2|10> and kills |00>, |11>, so the gate is the identity there and
    cos(2 theta) - i sin(2 theta) X on the span of |01>, |10>."""
    c, s = np.cos(2 * theta), np.sin(2 * theta)
    u = np.eye(4, dtype=np.complex128)
    u[1, 1] = u[2, 2] = c
    u[1, 2] = u[2, 1] = -1j * s
    return u


def neel_thetas(Lx, Ly):
    """Angles of Eq. initial_state giving |Neel> exactly in the oracle's product form:
    theta_j = pi (|1>) where (-1)^j = +1, 0 (|0>) elsewhere."""
    return np.array([np.pi if stag_sign(Ly, j) > 0 else 0.0 for j in range(Lx * Ly)])


# ------------------------------------------------------------------ state vector
def sv_apply_2q(psi, n, a, b, u):
    """Apply the 4 x 4 matrix u to qubits (a, b) (a the more significant index of u)."""
    t = psi.reshape((2,) * n)
    t = np.moveaxis(t, (a, b), (0, 1)).reshape(4, -1)
    t = (u @ t).reshape((2, 2) + (2,) * (n - 2))
    return np.moveaxis(t, (0, 1), (a, b)).reshape(-1)


def sv_neel(Lx, Ly):
    n = Lx * Ly
    idx = 0
    for j in range(n):
        if stag_sign(Ly, j) > 0:
            idx |= 1 << (n - 1 - j)
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[idx] = 1.0
    return psi


def sv_step(psi, Lx, Ly, g, dt):
    """One application of Eq. xy_trotter_step."""
    n = Lx * Ly
    bl = bonds(Lx, Ly)
    for (s, w) in LAYERS:
        u = gate(0.5 * g * dt * w)  # exp(-i w dt (g/2)(XX + YY))
        for (j, k, t) in bl:
            if t == s:
                psi = sv_apply_2q(psi, n, j, k, u)
    return psi


def sv_zstag(psi, Lx, Ly, alpha):
    """exp(-i alpha H_Z), H_Z = sum_j (-1)^j Z_j (diagonal)."""
    n = Lx * Ly
    z = sv._z_values(n).astype(np.float64)
    e = sum(stag_sign(Ly, j) * z[j] for j in range(n))
    return psi * np.exp(-1j * alpha * e)


def sv_observables(psi, Lx, Ly):
    """(<Z_tot>, <X_stag^2> of Eq. xy_signal, norm^2): <X_stag^2> = ||M psi||^2 / n^2 with
    M = sum_j (-1)^j X_j (Hermitian), <Z_tot> = (1/n) sum_j <Z_j>."""
    n = Lx * Ly
    p = np.abs(psi) ** 2
    norm = float(p.sum())
    z = sv._z_values(n).astype(np.float64)
    ztot = float((p * z.sum(axis=0)).sum() / (n * norm))
    xm = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    mpsi = np.zeros_like(psi)
    for j in range(n):
        mpsi += stag_sign(Ly, j) * sv.apply_1q(psi, n, j, xm)
    return ztot, float(np.vdot(mpsi, mpsi).real / (n * n * norm)), norm


def sv_run(Lx, Ly, steps, prep_steps, g=G_PAPER, dt=DT_PAPER, dtau=DTAU_PAPER):
    """Eq. xy_init with prep_steps Trotter steps of dtau, then `steps` quench steps of dt;
    per-step arrays (entry 0 = the initial state) and the final vector."""
    psi = sv_neel(Lx, Ly)
    for _ in range(prep_steps):
        psi = sv_step(psi, Lx, Ly, g, dtau)
    psi = sv_zstag(psi, Lx, Ly, np.pi / 8)
    rec = {"Z": [], "X2": []}
    for i in range(steps + 1):
        if i:
            psi = sv_step(psi, Lx, Ly, g, dt)
        z, x2, _ = sv_observables(psi, Lx, Ly)
        rec["Z"].append(z)
        rec["X2"].append(x2)
    return {k: np.array(v) for k, v in rec.items()}, psi


# ------------------------------------------------------------------ MPS
class XYMPS(mps.MPS):
    """The oracle MPS on the one-to-one row snake, started from |Neel>."""

    def __init__(self, Lx, Ly, chi):
        super().__init__(Lx, Ly, chi, 0.0)
        self.layout = blocks(Lx, Ly)
        self.n = Lx * Ly
        self.blocks = []
        for b in self.layout:
            v = np.zeros((1, 2, 1), dtype=np.complex128)
            v[0, 1 if stag_sign(Ly, b["qubits"][0]) > 0 else 0, 0] = 1.0
            self.blocks.append(v)
        self.centre = 0

    def gate_swap(self, gt, u):
        """The two-qubit gate u on sites p < q by SWAP routing: site q travels left next to site
        p (q - p - 1 two-site SWAP updates), u is applied in one two-site update of sites p, p+1,
        and the site travels back; every two-site update is a truncation (oracle.mps)."""
        p, q = gt[0], gt[1]
        self.move_centre(q)
        for m in range(q - 1, p, -1):
            self._two_site(m, swap=True, centre_left=True)
        self._two_site(p, gate=u, centre_left=False)
        for m in range(p + 1, q):
            self._two_site(m, swap=True, centre_left=False)
        self.centre = q

    def step(self, g, dt, sched):
        for (s, w) in LAYERS:
            u = gate(0.5 * g * dt * w)
            for gt in sched[s]:
                self.gate_swap(gt, u)

    def zstag(self, alpha):
        for p, b in enumerate(self.layout):
            w = stag_sign(self.Ly, b["qubits"][0])
            self.apply_local(p, np.diag(np.exp(-1j * alpha * w * np.array([1.0, -1.0]))))

    def x_stag2(self):
        """<X_stag^2> of Eq. xy_signal by the plain pairwise definition:
        (1/n^2) sum_{p, p'} w_p w_p' <X_p X_p'> (X_p^2 = I on the diagonal), normalised."""
        N = len(self.blocks)
        xm = np.array([[0, 1], [1, 0]], dtype=np.complex128)

        def transfer(E, A, op=None):
            Ak = A if op is None else np.einsum("st,ltr->lsr", op, A)
            return np.tensordot(np.tensordot(E, Ak, axes=([0], [0])), A.conj(), axes=([0, 1], [0, 1]))

        left = [np.ones((1, 1), dtype=np.complex128)]
        for p in range(N):
            left.append(transfer(left[-1], self.blocks[p]))
        norm = left[-1][0, 0].real
        right = [None] * (N + 1)
        right[N] = np.ones((1, 1), dtype=np.complex128)
        for p in range(N - 1, -1, -1):
            A = self.blocks[p]
            right[p] = np.tensordot(np.tensordot(A, right[p + 1], axes=([2], [0])), A.conj(), axes=([1, 2], [1, 2]))
        w = [stag_sign(self.Ly, b["qubits"][0]) for b in self.layout]
        tot = float(N) * norm  # the p = p' terms: w_p^2 <X_p^2> = 1 each
        for p in range(N):
            E = transfer(left[p], self.blocks[p], xm)
            for p2 in range(p + 1, N):
                E2 = transfer(E, self.blocks[p2], xm)
                tot += 2.0 * w[p] * w[p2] * np.einsum("ab,ab->", E2, right[p2 + 1]).real
                E = transfer(E, self.blocks[p2])
        return tot / (self.n * self.n * norm)


def run(Lx, Ly, chi, steps, prep_steps, g=G_PAPER, dt=DT_PAPER, dtau=DTAU_PAPER):
    """TEBD of Eq. xy_init and Eq. xy_trotter_step; per-step arrays (entry 0 = the initial
    state): Z (<Z_tot>), X2 (<X_stag^2>), F; plus truncation fidelities, bond dims, the MPS."""
    sched = schedule(Lx, Ly)
    m = XYMPS(Lx, Ly, chi)
    for _ in range(prep_steps):
        m.step(g, dtau, sched)
    m.zstag(np.pi / 8)
    rec = {"Z": [], "X2": [], "F": [], "gap": []}
    for i in range(steps + 1):
        if i:
            m.step(g, dt, sched)
        rec["gap"].append(min(m.cut_gaps) if m.cut_gaps else float("inf"))
        m.cut_gaps = []
        rec["Z"].append(m.observables()[0])
        rec["X2"].append(m.x_stag2())
        rec["F"].append(m.F)
    out = {k: np.array(v) for k, v in rec.items()}
    out["min_cut_gap"] = float(np.min(out["gap"]))
    out["fidelities"] = np.array(m.fidelities)
    out["bond_dims"] = m.bond_dims()
    out["mps"] = m
    return out
