"""The material constants the workloads hand to both the CUDA path and the
oracle are the paper's: each row of its material tables (appendix "Material
Parameters") and the simple damage constants of Sec. 4.3, kept as printed in
tests/golden/material_parameters.txt, against workloads' material records
(SI units).  CPU only."""
import os

import pytest

from paper_2210_04037_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
GIGA = 1e9

MATERIALS = {"CuBe": W.cube(), "Al-H32": W.al_h32(), "Steel": W.steel_304l_disk(),
             "U-Nb": W.u_nb()}
# table -> the record's keys of each column, and the columns given in GPa
COLUMNS = {
    "romenskii": (("rho0", "K0", "G0", "alpha", "beta", "Gamma0"), {"K0", "G0"}),
    "steinberg": (("rho0", "K0", "G0", "Gp", "alpha", "Gamma0", "Gamma1", "Gamma2", "gamma_s"),
                  {"K0", "G0"}),
    "johnson_cook": (("c1", "c2", "c3", "n_hard"), {"c1", "c2"}),
    "bonora": (("D_crit", "eps_t", "eps_c", "alpha_D", "poisson"), set()),
    "simple": (("Ddot0", "D_crit"), set()),
}


def rows():
    with open(os.path.join(HERE, "golden", "material_parameters.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                yield line[0], line[1], [float(v) for v in line[2:]]


def test_fixture_covers_every_table_row():
    seen = {(t, m) for t, m, _ in rows()}
    assert len(seen) == 12
    assert {t for t, _ in seen} == set(COLUMNS)


@pytest.mark.parametrize("table,name,values", list(rows()))
def test_workload_material_carries_the_printed_row(table, name, values):
    keys, giga = COLUMNS[table]
    m = MATERIALS[name]
    assert len(values) == len(keys)
    for k, v in zip(keys, values):
        want = v * GIGA if k in giga else v
        assert m[k] == pytest.approx(want, rel=1e-15, abs=0.0), (table, name, k)
    # the closure and models the row belongs to
    if table == "steinberg":
        assert m["shear_model"] == W.SHEAR_STEINBERG
    if table == "bonora":
        assert m["damage"] == 1
    if table == "simple":
        assert m["damage"] == 2
