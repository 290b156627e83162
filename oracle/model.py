"""TFIM model definitions (test infrastructure only; see oracle/__init__.py).

Supplemental Material, section "3D Transverse Field Ising Model": the same Hamiltonian on an
Lx x Ly x Lz cubic grid with open boundaries, the same product initial state, the temperatures
dtheta = 0, pi/9, 2 pi/9.  Reading where that section is silent: theta_min keeps its definition
asin(h / (d J)) with d = 6, the number of neighbours of a bulk site of the cubic lattice.

Sec. II, Eq. hamiltonian: H = J sum_<ij> Z_i Z_j + h sum_i X_i, nearest
neighbours with periodic boundaries on an Lx x Ly square lattice.
Sec. II, Eq. initial_state: |Psi(theta)> = prod_j (cos(theta/2)|0> + sin(theta/2)|1>).
Sec. II: theta_min = asin(h / (d J)) with d = 4 neighbours; theta = theta_min + dtheta;
the three "temperatures" dtheta = 0, 2 pi/9, 3 pi/9 at dt = 0.25, J = -1, h = 2.

Conventions (readings where the paper is silent):
* qubit (r, c) has global index r * Ly + c; |0> is the Z = +1 eigenstate;
* a Trotter layer is exp(-i dt H_part) written out literally: the X layer is
  prod_j exp(-i alpha X_j) with alpha = h dt / 2 (second order, Eq. trotter_step)
  or h dt (first order), the ZZ layer is prod_<ij> exp(-i phi Z_i Z_j) with
  phi = J dt -- no extra factor 1/2 on either angle;
* on a periodic side of length 2 the wrap bond coincides with the inner bond
  and is counted once.
"""
import math

J_PAPER = -1.0
H_PAPER = 2.0
DT_PAPER = 0.25
COORDINATION = 4  # neighbours of a site on the square lattice (the "d" of theta_min)

TEMPERATURES = {"low": 0.0, "mid": 2.0 * math.pi / 9.0, "high": 3.0 * math.pi / 9.0}
COORDINATION_3D = 6
TEMPERATURES_3D = {"low": 0.0, "mid": math.pi / 9.0, "high": 2.0 * math.pi / 9.0}


def theta_min(J=J_PAPER, h=H_PAPER, coordination=COORDINATION):
    """Sec. II: theta_min = asin(h / (d J)), the minimum of the mean-field energy."""
    return math.asin(h / (coordination * J))


def initial_theta(dtheta, J=J_PAPER, h=H_PAPER, coordination=COORDINATION):
    """Sec. II: theta = theta_min + dtheta."""
    return theta_min(J, h, coordination) + dtheta


def mean_field_energy_per_site(theta, J=J_PAPER, h=H_PAPER, coordination=COORDINATION):
    """<H>/n in the product state of Eq. initial_state: <Z> = cos theta, <X> = sin theta,
    and each site owns coordination/2 bonds."""
    return J * (coordination / 2.0) * math.cos(theta) ** 2 + h * math.sin(theta)


def layer_angles(J, h, dt, order):
    """Angles of the Trotter layers (Eq. trotter_step for order 2).

    Returns (alpha_x, phi_zz): the X layer is exp(-i alpha_x X) per qubit, applied
    twice per step for order 2 and once (before ZZ) for order 1; the ZZ layer is
    exp(-i phi_zz Z Z) per bond.
    """
    if order == 2:
        return 0.5 * h * dt, J * dt
    if order == 1:
        return h * dt, J * dt
    raise ValueError("trotter order must be 1 or 2")


def lattice_bonds(Lx, Ly):
    """Nearest-neighbour pairs (q1 < q2) with periodic boundaries, each bond once."""
    bonds = set()
    for r in range(Lx):
        for c in range(Ly):
            q = r * Ly + c
            for (rr, cc) in (((r + 1) % Lx, c), (r, (c + 1) % Ly)):
                q2 = rr * Ly + cc
                if q2 != q:
                    bonds.add((min(q, q2), max(q, q2)))
    return sorted(bonds)


def lattice_bonds_3d(Lx, Ly, Lz):
    """Nearest-neighbour pairs (q1 < q2) of the open Lx x Ly x Lz cubic grid; qubit (x, y, z) has
    the index (z Lx + x) Ly + y."""
    def q(x, y, z):
        return (z * Lx + x) * Ly + y

    bonds = []
    for z in range(Lz):
        for x in range(Lx):
            for y in range(Ly):
                for (xx, yy, zz) in ((x + 1, y, z), (x, y + 1, z), (x, y, z + 1)):
                    if xx < Lx and yy < Ly and zz < Lz:
                        bonds.append((q(x, y, z), q(xx, yy, zz)))
    return sorted(bonds)
