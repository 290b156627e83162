"""Exact state-vector Trotter simulator for <= 24 qubits (test infrastructure only).

Sec. II: Eq. initial_state, Eq. trotter_step (second order) and the first-order
product exp(-i dt H_ZZ) exp(-i dt H_X); observables Eq. Z_tot and Eq. z2_tot, and
<X_tot> = (1/n) sum_j <X_j> (the paper defines X_tot only for the XY model; this
is the TFIM reading).

The state is a complex128 vector over 2^n basis states, qubit q being axis q of
the (2,)*n reshape (qubit 0 most significant).  The ZZ layer is the exact diagonal
phase exp(-i phi E(z)) with E(z) = sum over bonds of z_i z_j.
"""
import numpy as np

from . import model

MAX_QUBITS = 24


def _z_values(n):
    """z_q(basis) = +1 if bit q is 0 else -1, as an (n, 2^n) int8 array."""
    idx = np.arange(2 ** n, dtype=np.int64)
    z = np.empty((n, 2 ** n), dtype=np.int8)
    for q in range(n):
        bit = (idx >> (n - 1 - q)) & 1
        z[q] = 1 - 2 * bit
    return z


def product_state(n, theta):
    """Eq. initial_state as a dense vector (theta: one angle, or one per qubit)."""
    if n > MAX_QUBITS:
        raise ValueError("state vector limited to %d qubits" % MAX_QUBITS)
    thetas = np.broadcast_to(np.asarray(theta, dtype=np.float64), (n,))
    psi = np.ones(1, dtype=np.complex128)
    for q in range(n):
        v = np.array([np.cos(thetas[q] / 2.0), np.sin(thetas[q] / 2.0)], dtype=np.complex128)
        psi = np.kron(psi, v)
    return psi


def apply_1q(psi, n, q, u):
    """Apply the 2x2 matrix u to qubit q."""
    t = psi.reshape((2,) * n)
    t = np.tensordot(u, t, axes=([1], [q]))
    t = np.moveaxis(t, 0, q)
    return t.reshape(-1)


def rx(alpha):
    """exp(-i alpha X)."""
    c, s = np.cos(alpha), np.sin(alpha)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def x_layer(psi, n, alpha):
    u = rx(alpha)
    for q in range(n):
        psi = apply_1q(psi, n, q, u)
    return psi


def zz_energy(Lx, Ly, Lz=None):
    """E(z) = sum_<ij> z_i z_j for every basis state (periodic 2D grid, or open 3D grid)."""
    n = Lx * Ly * (Lz or 1)
    z = _z_values(n).astype(np.int32)
    e = np.zeros(2 ** n, dtype=np.int32)
    bonds = model.lattice_bonds(Lx, Ly) if Lz is None else model.lattice_bonds_3d(Lx, Ly, Lz)
    for (a, b) in bonds:
        e += z[a] * z[b]
    return e


def zz_layer(psi, energy, phi):
    return psi * np.exp(-1j * phi * energy)


def observables(psi, n):
    """(<Z_tot>, <Z_tot^2>, <X_tot>, norm^2) by direct sums over the basis."""
    p = np.abs(psi) ** 2
    norm = p.sum()
    z = _z_values(n).astype(np.float64)
    m = z.sum(axis=0)
    ztot = float((p * m).sum() / (n * norm))
    z2 = float((p * m * m).sum() / (n * n * norm))
    t = psi.reshape((2,) * n)
    xs = 0.0
    for q in range(n):
        xs += np.vdot(t, np.flip(t, axis=q)).real
    return ztot, z2, float(xs / (n * norm)), float(norm)


def run(Lx, Ly, theta, J, h, dt, steps, order=2, Lz=None):
    """Trotter evolution; returns per-step arrays (step 0 = initial state) and psi."""
    n = Lx * Ly * (Lz or 1)
    alpha, phi = model.layer_angles(J, h, dt, order)
    energy = zz_energy(Lx, Ly, Lz)
    psi = product_state(n, theta)
    rec = {"Z": [], "Z2": [], "X": []}

    def record(v):
        z, z2, x, _ = observables(v, n)
        rec["Z"].append(z)
        rec["Z2"].append(z2)
        rec["X"].append(x)

    record(psi)
    for _ in range(steps):
        psi = x_layer(psi, n, alpha)
        psi = zz_layer(psi, energy, phi)
        if order == 2:
            psi = x_layer(psi, n, alpha)
        record(psi)
    return {k: np.array(v) for k, v in rec.items()}, psi
