"""C ABI and host logic, without a GPU: the library loads, exports every symbol the
header declares, and its host-only functions agree with the oracle's independent
layout / schedule and with the paper's gamma table."""
import json
import math
import os
import re
import subprocess

import pytest

from oracle import layout, model, rescale

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpsgb.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_23438_gb300 import build, lib as L
    build.build()
    L.load()
    return L


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mpsgb_[a-z0-9_]+)\s*\(", txt)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 20
    so = lib.load()
    for n in names:
        assert hasattr(so, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mpsgb_\w+)", out))
    assert set(names) <= exported
    assert set(lib.exported_symbols()) == set(names)


@pytest.mark.parametrize("grid", [(3, 3), (3, 4), (4, 4), (5, 6), (6, 6), (6, 8), (7, 8)])
def test_schedule_matches_oracle(lib, grid):
    info = lib.schedule_info(*grid)
    nb, nintra, dist, ntr = layout.census(*grid)
    assert info["zz_bonds"] == nb and info["intra"] == nintra and info["truncations"] == ntr
    assert info["blocks"] == 2 * grid[0]
    _, inter = layout.schedule(*grid)
    assert lib.schedule_gates(*grid) == [tuple(g) for g in inter]


@pytest.mark.parametrize("dims", [(2, 2, 2), (2, 3, 4), (3, 3, 4), (4, 4, 4), (3, 4, 2)])
def test_3d_schedule_matches_oracle(lib, dims):
    # open cubic grid, one qubit per site along the 3D snake: the library's gate list (positions,
    # qubits, bit positions) equals the oracle's, element by element
    Lx, Ly, Lz = dims
    cfg = lib.config(Lx, Ly, 16, 0.1, lattice=lib.LATTICE_3D_SITES, Lz=Lz)
    _, inter = layout.schedule_3d(Lx, Ly, Lz)
    assert lib.schedule_gates(cfg) == [tuple(g) for g in inter]
    info = lib.schedule_info(cfg)
    assert info["blocks"] == Lx * Ly * Lz and info["intra"] == 0 and info["dmax"] == 2
    assert info["inter"] == len(inter) and info["truncations"] == sum(g[1] - g[0] for g in inter)
    # 2D configs give the same answers through either query
    c2 = lib.config(5, 6, 16, 0.1)
    assert lib.schedule_gates(c2) == lib.schedule_gates(5, 6)
    # footprint: chi capped by the largest exact bound (2^(n/2)), d = 2, one site per qubit
    chi = min(16, 2 ** (Lx * Ly * Lz // 2))
    assert lib.footprint_bytes(cfg) == chi * chi * 2 * Lx * Ly * Lz * 16


@pytest.mark.parametrize("dims", [(2, 2), (3, 4), (4, 4), (5, 6), (6, 6)])
def test_2d_sites_schedule_matches_oracle(lib, dims):
    # open grid, one qubit per site along the row snake (the XY workload's lattice): the library's
    # gate list equals the oracle's bond sets A..D merged in (first site, second site) order
    from oracle import xy
    Lx, Ly = dims
    cfg = lib.xy_config(Lx, Ly, 16, 1.0, 0.1)
    sched = xy.schedule(Lx, Ly)
    merged = sorted([g for v in sched.values() for g in v], key=lambda g: (g[0], g[1], g[2], g[3]))
    assert lib.schedule_gates(cfg) == [tuple(g) for g in merged]
    info = lib.schedule_info(cfg)
    assert info["blocks"] == Lx * Ly and info["intra"] == 0 and info["dmax"] == 2
    assert info["inter"] == Lx * (Ly - 1) + (Lx - 1) * Ly


def test_host_formulas(lib):
    assert abs(lib.initial_theta(-1.0, 2.0, 0.0) - model.theta_min()) < 1e-15
    assert abs(lib.initial_theta(-1.0, 2.0, 0.0, lattice=lib.LATTICE_2D_GROUPED) - model.theta_min()) < 1e-15
    t3 = model.initial_theta(math.pi / 9, coordination=model.COORDINATION_3D)
    assert abs(lib.initial_theta(-1.0, 2.0, math.pi / 9, lattice=lib.LATTICE_3D_SITES) - t3) < 1e-15
    assert math.isnan(lib.initial_theta(-1.0, 2.0, 0.0, lattice=5))
    for t, name in enumerate(("low", "mid", "high")):
        for chi, n in [(64, 30), (1024, 48), (4096, 56)]:
            assert abs(lib.gamma_fit(t, chi, n) - rescale.gamma_fit(name, chi, n)) < 1e-15
    assert math.isnan(lib.gamma_fit(3, 64, 30))
    for t, name in enumerate(("low", "mid", "high")):
        for chi, n in [(64, 36), (256, 64), (1024, 36)]:
            g3 = lib.gamma_fit(t, chi, n, lattice=lib.LATTICE_3D_SITES)
            assert abs(g3 - rescale.gamma_fit(name, chi, n, three_d=True)) < 1e-15
            assert lib.gamma_fit(t, chi, n, lattice=lib.LATTICE_2D_GROUPED) == lib.gamma_fit(t, chi, n)
    assert math.isnan(lib.gamma_fit(0, 64, 36, lattice=lib.LATTICE_2D_SITES))
    z, z2 = lib.rescale(0.3, 0.2, 0.5, 0.7)
    assert abs(z - rescale.rescale_z(0.3, 0.5)) < 1e-16
    assert abs(z2 - rescale.rescale_z2(0.2, 0.5, 0.7)) < 1e-16


def test_footprint(lib):
    # chi^2 * dmax * blocks * element size (complex128 in the FP64 form)
    assert lib.footprint_bytes(lib.config(6, 8, 1024, 0.1)) == 1024 ** 2 * 16 * 12 * 16
    assert lib.footprint_bytes(lib.config(6, 8, 1024, 0.1, prec="fp32")) == 1024 ** 2 * 16 * 12 * 8
    # chi above every bond bound is capped by the largest bound (3x4: 64)
    assert lib.footprint_bytes(lib.config(3, 4, 1000, 0.1)) == 64 ** 2 * 4 * 6 * 16


def test_invalid_arguments_rejected_on_host(lib):
    for cfg in [lib.config(1, 4, 16, 0.1), lib.config(3, 4, 0, 0.1), lib.config(3, 4, 16, float("nan")),
                lib.config(3, 4, 16, 0.1, prec=7), lib.config(3, 40, 16, 0.1),
                lib.config(3, 4, 16, 0.1, Lz=2), lib.config(3, 4, 16, 0.1, lattice=3),
                lib.config(3, 4, 16, 0.1, model=2), lib.config(3, 4, 16, 0.1, model=lib.MODEL_XY),
                lib.config(3, 4, 16, 0.1, model=lib.MODEL_XY, lattice=lib.LATTICE_2D_SITES),
                lib.config(3, 4, 16, 0.1, model=lib.MODEL_XY, lattice=lib.LATTICE_2D_SITES, route=lib.ROUTE_SWAP,
                           order=1),
                lib.config(17, 4, 16, 0.1, lattice=lib.LATTICE_2D_SITES),
                lib.config(3, 3, 16, 0.1, lattice=1, Lz=1), lib.config(9, 9, 16, 0.1, lattice=1, Lz=9)]:
        with pytest.raises(lib.MpsgbError) as e:
            lib.MPS(cfg)
        assert e.value.status == -1
    with pytest.raises(lib.MpsgbError):
        lib.schedule_info(2, 1)
