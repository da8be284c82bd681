"""Long-run bulk statistics: the oracle, the plain FP64 form and the chosen form (voxel
positions + FP32 arithmetic, delayed audited detection) agree on the packing fraction and
the mean coordination number within 0.5%.

Trajectories of many colliding spheres separate once rounding differs, so these runs are
compared through bulk quantities: each is averaged over samples taken at fixed steps, in
a window at least 3 r_max from every wall."""
import numpy as np
import pytest

import oracle
from oracle import statistics as S
from paper_2311_04648_gb300 import dem
from paper_2311_04648_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 0.005
MARGIN = 6e-5      # margin of the chosen form


def _column():
    # the 4M settling column's generator restricted to a 30 mm wide column (20k spheres)
    sc = W.settling_column(n=20000, column_width=0.03)
    r = sc.r_max
    top = float(np.max(sc.x[:, 2]))
    lo = np.array([sc.box_lo[0] + 3 * r, sc.box_lo[1] + 3 * r, sc.box_lo[2] + 3 * r])
    hi = np.array([sc.box_hi[0] - 3 * r, sc.box_hi[1] - 3 * r, 0.5 * top])
    return sc, lo, hi, list(range(1000, 5001, 500))


def _dense():
    # a jittered lattice spaced below the contact distance: about five contacts a sphere
    sc = W.dense_lattice(n=20000, seed=7)
    r = sc.r_max
    return sc, sc.box_lo + 3 * r, sc.box_hi - 3 * r, list(range(500, 2001, 250))


def _sample_oracle(sc, lo, hi, at):
    o = oracle.OracleWorld(sc, cell_list=True)
    phi, z, done = [], [], 0
    for s in at:
        assert o.step(s - done) == 0
        done = s
        p = o.sphere_positions()
        _, _, cs = o.eval()
        phi.append(S.packing_fraction(p, o.rad, lo, hi))
        z.append(S.coordination(p, cs["i"], cs["j"], lo, hi)[0])
    return np.mean(phi), np.mean(z)


def _sample_gpu(w, lo, hi, at):
    phi, z, done = [], [], 0
    for s in at:
        w.step(s - done)
        done = s
        p, r = w.sphere_positions()
        c = w.contacts()
        touch = c["overlap"] > 0
        phi.append(S.packing_fraction(p, r, lo, hi))
        z.append(S.coordination(p, c["i"][touch], c["j"][touch], lo, hi)[0])
    return np.mean(phi), np.mean(z)


@pytest.mark.parametrize("case", ["column", "dense"])
def test_long_run_statistics_agree(case):
    sc, lo, hi, at = _column() if case == "column" else _dense()
    plain = dem.World.from_scene(sc, precision="fp64", schedule="every_step")
    chosen = dem.World.from_scene(sc, precision="voxel_fp32", schedule="velocity_bound", margin=MARGIN,
                                  margin_max=MARGIN)
    try:
        phi_p, z_p = _sample_gpu(plain, lo, hi, at)
        phi_c, z_c = _sample_gpu(chosen, lo, hi, at)
    finally:
        plain.close()
        chosen.close()
    phi_o, z_o = _sample_oracle(sc, lo, hi, at)
    print(f"{case}: packing oracle {phi_o:.6f} plain {phi_p:.6f} chosen {phi_c:.6f}; "
          f"coordination oracle {z_o:.5f} plain {z_p:.5f} chosen {z_c:.5f}")
    assert z_o > 0.02 and phi_o > 0.2
    assert abs(phi_p - phi_o) <= TOL * phi_o
    assert abs(z_p - z_o) <= TOL * z_o
    assert abs(phi_c - phi_p) <= TOL * phi_p
    assert abs(z_c - z_p) <= TOL * z_p
