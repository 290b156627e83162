"""Plain MPS TEBD of the grouped-qubit TFIM (test infrastructure only).

Sec. III: the circuit U(dt)^s is applied gate by gate; after each gate the MPS is
brought back to canonical form and truncated by singular-value decomposition to at
most chi, renormalised to unit norm, and the truncation fidelity is kept
separately; F_MPS(s) is the product of all truncation fidelities up to step s.
The orthogonality centre is moved to the gate's bond before the decomposition.
Qubits are grouped into blocks (oracle.layout); a gate inside a block updates the
block tensor and leaves bond dimensions unchanged; a gate between blocks is applied
as a rank-2 MPO (exp(-i phi Z_i Z_j) = cos(phi) I I - i sin(phi) Z_i Z_j), which
doubles every virtual bond between the two blocks.

Plain definition used for an inter-block gate on blocks p < q (centre on p):
  1. apply the MPO: block p gets the two branches [cos(phi) A, -i sin(phi) Z_i A]
     on its right bond, blocks strictly between get C (x) delta_2, block q gets
     [B ; Z_j B] on its left bond;
  2. right-canonicalise blocks q .. p+1 by LQ decompositions;
  3. for bonds p .. q-1 in order: SVD of the current centre block reshaped to
     (left * d, right) with numpy.linalg.svd (LAPACK, FP64); keep the
     k = min(chi, numerical rank) largest singular values; the truncation fidelity
     is f = sum_kept s^2 / sum_all s^2; renormalise the kept values to unit norm and
     push diag(s) V^H into the next block.
Numerical rank follows numpy's matrix_rank rule: s > s_max * max(shape) * eps.
Ties at the chi cut are broken by LAPACK's order (several truncations are then
equally correct; tests compare only gauge-invariant quantities there).

Blocks are complex128 arrays of shape (left, d, right).
"""
import numpy as np

from . import layout, model


def _rank_keep(s, shape, chi):
    if s.size == 0:
        return 0
    tol = s[0] * max(shape) * np.finfo(np.float64).eps
    return int(min(chi, np.count_nonzero(s > tol)))


class MPS:
    """Grouped-qubit MPS with an explicit orthogonality centre (a block index)."""

    def __init__(self, Lx, Ly, chi, theta, Lz=None):
        """theta: the angle of Eq. initial_state, or one angle per qubit (global qubit index).
        Lz: None for the grouped 2D grid; a layer count for the 3D one-to-one mapping."""
        self.Lx, self.Ly, self.Lz, self.chi = Lx, Ly, Lz, chi
        self.layout = layout.blocks(Lx, Ly) if Lz is None else layout.blocks_3d(Lx, Ly, Lz)
        self.n = sum(len(b["qubits"]) for b in self.layout)
        thetas = np.broadcast_to(np.asarray(theta, dtype=np.float64), (self.n,))
        self.blocks = []
        for b in self.layout:
            phys = np.ones(1, dtype=np.complex128)
            for q in b["qubits"]:
                v = np.array([np.cos(thetas[q] / 2.0), np.sin(thetas[q] / 2.0)], dtype=np.complex128)
                phys = np.kron(phys, v)  # first qubit = most significant bit
            self.blocks.append(phys.reshape(1, b["d"], 1).copy())
        self.centre = 0
        self.F = 1.0
        self.fidelities = []  # every truncation fidelity f, in order
        self.kept_norms = []  # sum of kept s^2 at every truncation (before renormalising)
        self.cut_gaps = []  # (s_k-1 - s_k) / s_0 at every truncation that discarded something

    # ---------------------------------------------------------------- gauge moves
    def _qr_right(self, m):
        """Move the centre from block m to m+1 by QR (block m becomes left-isometric)."""
        A = self.blocks[m]
        l, d, r = A.shape
        Q, R = np.linalg.qr(A.reshape(l * d, r))
        self.blocks[m] = Q.reshape(l, d, Q.shape[1])
        self.blocks[m + 1] = np.tensordot(R, self.blocks[m + 1], axes=([1], [0]))

    def _lq_left(self, m):
        """Move the centre from block m to m-1 by LQ (block m becomes right-isometric)."""
        B = self.blocks[m]
        l, d, r = B.shape
        Q, R = np.linalg.qr(B.reshape(l, d * r).conj().T)
        L = R.conj().T
        self.blocks[m] = Q.conj().T.reshape(Q.shape[1], d, r)
        self.blocks[m - 1] = np.tensordot(self.blocks[m - 1], L, axes=([2], [0]))

    def move_centre(self, target):
        while self.centre < target:
            self._qr_right(self.centre)
            self.centre += 1
        while self.centre > target:
            self._lq_left(self.centre)
            self.centre -= 1

    # ---------------------------------------------------------------- local gates
    def apply_local(self, p, u):
        """Apply a d x d unitary to the physical leg of block p (no truncation)."""
        self.blocks[p] = np.einsum("st,ltr->lsr", u, self.blocks[p])

    @staticmethod
    def _zdiag(k, t):
        """z of bit t (0 = most significant) over the 2^k physical states."""
        s = np.arange(2 ** k)
        return 1.0 - 2.0 * ((s >> (k - 1 - t)) & 1)

    def x_layer(self, alpha):
        """prod_j exp(-i alpha X_j), block by block."""
        c, s = np.cos(alpha), np.sin(alpha)
        r1 = np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
        for p, b in enumerate(self.layout):
            u = np.ones((1, 1), dtype=np.complex128)
            for _ in b["qubits"]:
                u = np.kron(u, r1)
            self.apply_local(p, u)

    def zz_intra(self, phi, intra):
        """exp(-i phi Z_t Z_u) for every ZZ pair inside a block (diagonal)."""
        for p, pairs in enumerate(intra):
            if not pairs:
                continue
            k = len(self.layout[p]["qubits"])
            e = np.zeros(2 ** k)
            for (t, u) in pairs:
                e += self._zdiag(k, t) * self._zdiag(k, u)
            self.apply_local(p, np.diag(np.exp(-1j * phi * e)))

    # ---------------------------------------------------------------- inter-block gate
    def zz_inter(self, gate, phi):
        """One inter-block exp(-i phi Z_i Z_j) with the MPO + SVD sweep of the module docstring."""
        p, q, _, _, ti, tj = gate
        self.move_centre(p)
        ki = len(self.layout[p]["qubits"])
        kj = len(self.layout[q]["qubits"])
        zi = self._zdiag(ki, ti)
        zj = self._zdiag(kj, tj)
        # 1. MPO application (bond index of the MPO is the slow index of the new bond)
        A = self.blocks[p]
        A2 = np.concatenate([np.cos(phi) * A, (-1j * np.sin(phi)) * zi[None, :, None] * A], axis=2)
        self.blocks[p] = A2
        for m in range(p + 1, q):
            C = self.blocks[m]
            l, d, r = C.shape
            C2 = np.zeros((2 * l, d, 2 * r), dtype=np.complex128)
            C2[:l, :, :r] = C
            C2[l:, :, r:] = C
            self.blocks[m] = C2
        B = self.blocks[q]
        self.blocks[q] = np.concatenate([B, zj[None, :, None] * B], axis=0)
        # 2. right-canonicalise q .. p+1
        for m in range(q, p, -1):
            self._lq_left(m)
        # 3. SVD sweep p .. q-1
        for m in range(p, q):
            M = self.blocks[m]
            l, d, r = M.shape
            U, s, Vh = np.linalg.svd(M.reshape(l * d, r), full_matrices=False)
            k = _rank_keep(s, (l * d, r), self.chi)
            tot = float(np.sum(s * s))
            kept = float(np.sum(s[:k] ** 2))
            f = kept / tot
            if k < len(s) and s[k] > 0:
                self.cut_gaps.append((s[k - 1] - s[k]) / s[0])
            self.F *= f
            self.fidelities.append(f)
            self.kept_norms.append(kept)
            sk = s[:k] / np.sqrt(kept)
            self.blocks[m] = U[:, :k].reshape(l, d, k)
            self.blocks[m + 1] = np.tensordot(sk[:, None] * Vh[:k], self.blocks[m + 1], axes=([1], [0]))
        self.centre = q

    # ---------------------------------------------------------------- SWAP routing
    def _two_site(self, m, swap=False, phase=None, centre_left=True, gate=None):
        """Two-site update of blocks m, m+1 (the centre on one of them): theta = A B as a dense
        (left, d_m, d_m+1, right) tensor, optionally with a diagonal two-qubit phase on the two
        physical indices or with the two physical legs exchanged (a SWAP of the blocks), then the
        SVD of theta as a (left * d) x (d' * right) matrix with numpy.linalg.svd, truncated like
        the MPO sweep (min(chi, numerical rank) values, f = kept / total, renormalised).  The
        kept singular values go into block m (centre_left) or block m+1.  `gate`: a general
        (d_m d_m+1) x (d_m d_m+1) matrix on the two physical indices instead of a phase."""
        A, B = self.blocks[m], self.blocks[m + 1]
        l, da, _ = A.shape
        _, db, r = B.shape
        th = np.tensordot(A, B, axes=([2], [0]))  # (l, da, db, r)
        if phase is not None:
            th = th * phase[None, :, :, None]
        if gate is not None:
            th = np.einsum("xy,lyr->lxr", gate, th.reshape(l, da * db, r)).reshape(l, da, db, r)
        if swap:
            th = th.transpose(0, 2, 1, 3)
            da, db = db, da
        M = th.reshape(l * da, db * r)
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        k = _rank_keep(s, M.shape, self.chi)
        tot = float(np.sum(s * s))
        kept = float(np.sum(s[:k] ** 2))
        f = kept / tot
        if k < len(s) and s[k] > 0:
            self.cut_gaps.append((s[k - 1] - s[k]) / s[0])
        self.F *= f
        self.fidelities.append(f)
        self.kept_norms.append(kept)
        sk = s[:k] / np.sqrt(kept)
        if centre_left:
            self.blocks[m] = (U[:, :k] * sk[None, :]).reshape(l, da, k)
            self.blocks[m + 1] = Vh[:k].reshape(k, db, r)
        else:
            self.blocks[m] = U[:, :k].reshape(l, da, k)
            self.blocks[m + 1] = (sk[:, None] * Vh[:k]).reshape(k, db, r)
        if swap:
            self.layout[m], self.layout[m + 1] = self.layout[m + 1], self.layout[m]

    def zz_inter_swap(self, gate, phi):
        """One inter-block exp(-i phi Z_i Z_j) by SWAP routing: block q is swapped leftwards next
        to block p (q - p - 1 two-site SWAP updates, centre travelling left), the gate is applied
        as a diagonal phase in one two-site update of blocks p and p+1, and the block is swapped
        back (centre travelling right).  Every two-site update is an SVD truncation, so a gate of
        block distance k costs 2 (k - 1) + 1 of them.  Ends with the centre on block q."""
        p, q, _, _, ti, tj = gate
        self.move_centre(q)
        for m in range(q - 1, p, -1):
            self._two_site(m, swap=True, centre_left=True)
        zi = self._zdiag(len(self.layout[p]["qubits"]), ti)
        zj = self._zdiag(len(self.layout[p + 1]["qubits"]), tj)
        self._two_site(p, phase=np.exp(-1j * phi * np.outer(zi, zj)), centre_left=False)
        for m in range(p + 1, q):
            self._two_site(m, swap=True, centre_left=False)
        self.centre = q

    # ---------------------------------------------------------------- observables
    def bond_dims(self):
        return [b.shape[2] for b in self.blocks[:-1]]

    def to_statevector(self):
        """Contract to a dense vector with qubit order r * Ly + c (qubit 0 most significant)."""
        t = self.blocks[0]
        for b in self.blocks[1:]:
            t = np.tensordot(t, b, axes=([t.ndim - 1], [0]))
        t = t.reshape(t.shape[1:-1])  # drop the unit boundary bonds
        shape, order = [], []
        for b in self.layout:
            for q in b["qubits"]:
                shape.append(2)
                order.append(q)
        t = t.reshape(shape)
        perm = np.argsort(order)
        return np.transpose(t, perm).reshape(-1)

    def _block_ops(self, p):
        """Diagonal m_p(s) = sum_{j in block} z_j(s) and the off-diagonal x_p = sum_j X_j."""
        k = len(self.layout[p]["qubits"])
        d = 2 ** k
        m = np.zeros(d)
        x = np.zeros((d, d))
        s = np.arange(d)
        for t in range(k):
            m += self._zdiag(k, t)
            x[s, s ^ (1 << (k - 1 - t))] = 1.0
        return m, x

    def observables(self):
        """(<Z_tot>, <Z_tot^2>, <X_tot>, norm^2) by environment contraction.

        Plain definition, no canonical form assumed: <Z_tot^2> = (1/n^2) sum_{b,b'} <m_b m_b'>
        where m_b is the block's total Z; pairs are contracted one by one.
        """
        N = len(self.blocks)

        def transfer(E, A, op=None):
            # E: (l, l') left environment (ket index, bra index); op: d x d acting on the ket
            Ak = A if op is None else np.einsum("st,ltr->lsr", op, A)
            T = np.tensordot(E, Ak, axes=([0], [0]))  # (b, s, r)
            return np.tensordot(T, A.conj(), axes=([0, 1], [0, 1]))  # (r, q)

        ops = [self._block_ops(p) for p in range(N)]
        left = [np.ones((1, 1), dtype=np.complex128)]
        for p in range(N):
            left.append(transfer(left[-1], self.blocks[p]))
        norm = left[-1][0, 0].real
        right = [None] * (N + 1)
        right[N] = np.ones((1, 1), dtype=np.complex128)
        for p in range(N - 1, -1, -1):
            A = self.blocks[p]
            T = np.tensordot(A, right[p + 1], axes=([2], [0]))  # (a, s, q)
            right[p] = np.tensordot(T, A.conj(), axes=([1, 2], [1, 2]))  # (a, b)

        def close(E, p):
            return np.einsum("ab,ab->", E, right[p]).real

        ztot = 0.0
        xtot = 0.0
        z2 = 0.0
        for p in range(N):
            m, x = ops[p]
            ztot += close(transfer(left[p], self.blocks[p], np.diag(m)), p + 1)
            xtot += close(transfer(left[p], self.blocks[p], x), p + 1)
            z2 += close(transfer(left[p], self.blocks[p], np.diag(m * m)), p + 1)
            E = transfer(left[p], self.blocks[p], np.diag(m))
            for p2 in range(p + 1, N):
                E2 = transfer(E, self.blocks[p2], np.diag(ops[p2][0]))
                z2 += 2.0 * close(E2, p2 + 1)
                E = transfer(E, self.blocks[p2])
        n = self.n
        return ztot / (n * norm), z2 / (n * n * norm), xtot / (n * norm), norm

    def singular_values(self, bond):
        """Schmidt values across bond `bond` (between blocks bond and bond+1)."""
        saved = ([b.copy() for b in self.blocks], self.centre)
        self.move_centre(bond)
        A = self.blocks[bond]
        l, d, r = A.shape
        s = np.linalg.svd(A.reshape(l * d, r), compute_uv=False)
        self.blocks, self.centre = saved
        return s


def random_canonical(Lx, Ly, chi, seed, decay=None, centre=0, Lz=None, sites=None):
    """Seeded random MPS with every bond at min(chi, bound), in canonical form with the
    orthogonality centre on block `centre`, unit norm.  Entries are complex normal; with `decay`
    every block is scaled by exp(-b / decay) along its right bond index b, so that the Schmidt
    spectra fall off over the bond (a uniformly random state has nearly flat spectra).  The gauge
    moves are this module's QR / LQ steps.  An input generator for generic states: it computes
    nothing of the method and has no pin of its own (its outputs are checked for canonical form
    and norm where they are used).  Lz: layer count of the open 3D grid (one qubit per site);
    sites: an explicit list of sites in MPS order (dicts with "qubits" and "d"), e.g. oracle.xy.blocks."""
    rng = np.random.default_rng(seed)
    m = MPS(Lx, Ly, chi, 0.3, Lz=Lz)
    if sites is not None:
        m.layout = [dict(b) for b in sites]
        m.n = sum(len(b["qubits"]) for b in sites)
    ds = [b["d"] for b in m.layout]
    bd = [1] + [int(min(chi, b)) for b in layout.bond_bounds(Lx, Ly, m.layout)] + [1]
    blocks = []
    for i in range(len(ds)):
        shape = (bd[i], ds[i], bd[i + 1])
        b = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        if decay is not None:
            b *= np.exp(-np.arange(bd[i + 1]) / decay)[None, None, :]
        blocks.append(b)
    m.blocks = blocks
    m.centre = len(ds) - 1
    m.move_centre(0)
    m.blocks[0] /= np.linalg.norm(m.blocks[0])
    m.move_centre(centre)
    return m


def run(Lx, Ly, chi, theta, J, h, dt, steps, order=2, record_spectra=False, route="mpo", Lz=None):
    """TEBD run of Eq. trotter_step (order 2) or X-then-ZZ (order 1); inter-block gates by the MPO
    sweep (route "mpo", Sec. III) or by SWAP routing (route "swap").  Lz: None for the grouped 2D
    grid, else the layer count of the open 3D grid with one qubit per site.

    Returns a dict with per-step arrays (entry 0 = initial state): Z, Z2, X, F, plus the
    list of truncation fidelities, final bond dims and the MPS itself.
    """
    alpha, phi = model.layer_angles(J, h, dt, order)
    intra, inter = layout.schedule(Lx, Ly) if Lz is None else layout.schedule_3d(Lx, Ly, Lz)
    psi = MPS(Lx, Ly, chi, theta, Lz=Lz)
    rec = {"Z": [], "Z2": [], "X": [], "F": [], "spectra": [], "gap": []}

    def record():
        # smallest relative gap at any cut since the previous record (inf if nothing was cut)
        rec["gap"].append(min(psi.cut_gaps) if psi.cut_gaps else float("inf"))
        psi.cut_gaps = []
        z, z2, x, _ = psi.observables()
        rec["Z"].append(z)
        rec["Z2"].append(z2)
        rec["X"].append(x)
        rec["F"].append(psi.F)
        if record_spectra:
            rec["spectra"].append([psi.singular_values(m) for m in range(len(psi.blocks) - 1)])

    record()
    for _ in range(steps):
        psi.x_layer(alpha)
        psi.zz_intra(phi, intra)
        for g in inter:
            if route == "swap":
                psi.zz_inter_swap(g, phi)
            else:
                psi.zz_inter(g, phi)
        if order == 2:
            psi.x_layer(alpha)
        record()
    out = {k: np.array(v) for k, v in rec.items() if k != "spectra"}
    out["spectra"] = rec["spectra"]
    out["fidelities"] = np.array(psi.fidelities)
    out["kept_norms"] = np.array(psi.kept_norms)
    out["min_cut_gap"] = float(np.min(out["gap"]))
    out["bond_dims"] = psi.bond_dims()
    out["mps"] = psi
    return out
