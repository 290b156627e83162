"""Grouped-qubit MPS layout and gate schedule (test infrastructure only).

Sec. III and Fig. mps_drawing: the qubits of each row are split into two
groups, each group is fused into one MPS block, and blocks are ordered along a
snake (Sec. "MPS Ordering" of the Supplemental Material).

Readings where the paper is silent:
* group 0 of a row holds the columns c < ceil(Ly/2), group 1 the rest;
* MPS position of block (r, g) is 2r + g for even r and 2r + 1 - g for odd r
  (rows alternate direction);
* inside a block the qubits are ordered by column, the first one being the most
  significant bit of the physical index (big-endian); bit 0 is |0>, Z = +1;
* in-block ZZ gates need no truncation; inter-block gates are applied one
  two-qubit gate at a time, in the order sorted by
  (first block position, second block position, qubit in first block, qubit in second block).
"""
from . import model

# 3D variant (Supplemental Material, 3D TFIM section and Fig. 3D_snake): one qubit per MPS site.
# Reading of the snake where the figure is not reproduced: layer z = 0, 1, ... in turn; in layer z
# the rows x run 0 .. Lx-1 for even z and Lx-1 .. 0 for odd z; the k-th row visited overall runs
# y = 0 .. Ly-1 for even k and Ly-1 .. 0 for odd k.  Consecutive sites are then lattice neighbours.


def blocks(Lx, Ly):
    """Blocks in MPS order: list of dicts {row, group, qubits (global, big-endian), d}."""
    h0 = (Ly + 1) // 2
    out = [None] * (2 * Lx)
    for r in range(Lx):
        for g in range(2):
            cols = list(range(0, h0)) if g == 0 else list(range(h0, Ly))
            pos = 2 * r + g if r % 2 == 0 else 2 * r + 1 - g
            out[pos] = {"row": r, "group": g, "qubits": [r * Ly + c for c in cols],
                        "d": 2 ** len(cols)}
    return out


def blocks_3d(Lx, Ly, Lz):
    """Sites of the 3D one-to-one mapping in MPS order: list of dicts {xyz, qubits, d = 2}."""
    out = []
    k = 0
    for z in range(Lz):
        for i in range(Lx):
            x = i if z % 2 == 0 else Lx - 1 - i
            for j in range(Ly):
                y = j if k % 2 == 0 else Ly - 1 - j
                out.append({"xyz": (x, y, z), "qubits": [(z * Lx + x) * Ly + y], "d": 2})
            k += 1
    return out


def qubit_home(Lx, Ly, blks=None):
    """Map global qubit -> (MPS position, bit position from the most significant end)."""
    home = {}
    for p, b in enumerate(blks if blks is not None else blocks(Lx, Ly)):
        for t, q in enumerate(b["qubits"]):
            home[q] = (p, t)
    return home


def bond_bounds(Lx, Ly, blks=None):
    """Exact bond dimension bound of bond m (between blocks m and m+1): the smaller of
    the Hilbert-space dimensions on either side."""
    ds = [b["d"] for b in (blks if blks is not None else blocks(Lx, Ly))]
    bounds = []
    for m in range(len(ds) - 1):
        left = 1
        for d in ds[: m + 1]:
            left *= d
        right = 1
        for d in ds[m + 1:]:
            right *= d
        bounds.append(min(left, right))
    return bounds


def schedule(Lx, Ly):
    """Split the ZZ bonds into in-block pairs and the ordered list of inter-block gates.

    Returns (intra, inter):
      intra[p] = list of (t, u) bit positions of ZZ pairs inside block p;
      inter    = list of (p, q, qi, qj, ti, tj) with p < q the block positions,
                 qi/qj the global qubits and ti/tj their bit positions.
    """
    return _split_bonds(qubit_home(Lx, Ly), 2 * Lx, model.lattice_bonds(Lx, Ly))


def schedule_3d(Lx, Ly, Lz):
    """(intra, inter) of the 3D one-to-one mapping, as schedule(): every bond is an inter-site gate."""
    return _split_bonds(qubit_home(0, 0, blocks_3d(Lx, Ly, Lz)), Lx * Ly * Lz, model.lattice_bonds_3d(Lx, Ly, Lz))


def _split_bonds(home, nblk, bonds):
    intra = [[] for _ in range(nblk)]
    inter = []
    for (q1, q2) in bonds:
        p1, t1 = home[q1]
        p2, t2 = home[q2]
        if p1 == p2:
            intra[p1].append((min(t1, t2), max(t1, t2)))
        else:
            if p1 > p2:
                p1, p2, q1, q2, t1, t2 = p2, p1, q2, q1, t2, t1
            inter.append((p1, p2, q1, q2, t1, t2))
    inter.sort(key=lambda g: (g[0], g[1], g[2], g[3]))
    return intra, inter


def census(Lx, Ly):
    """Per-step counts: (#bonds, #in-block, {distance: #gates}, #bond truncations)."""
    intra, inter = schedule(Lx, Ly)
    dist = {}
    for g in inter:
        k = g[1] - g[0]
        dist[k] = dist.get(k, 0) + 1
    n_intra = sum(len(x) for x in intra)
    return (n_intra + len(inter), n_intra, dict(sorted(dist.items())),
            sum(k * c for k, c in dist.items()))
