"""Pins of the oracle's coordination zones against eq. (z), eq. (zeta) and Table I."""
import math
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_pc.txt")


def load_table1():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        label, z, zeta, pc = line.split()
        mask = sum(1 << (int(k) - 1) for k in label.split(","))
        rows.append((label, mask, int(z), float(zeta), float(pc)))
    return rows


def corrected_table1():
    """Table I with the two misprinted labels swapped back (their z is fixed by eq. z)."""
    rows = load_table1()
    by_label = {r[0]: r for r in rows}
    a, b = by_label["1,3,4,5,7"], by_label["1,3,4,6,7"]
    fixed = []
    for r in rows:
        if r[0] == "1,3,4,5,7":
            r = (r[0], r[1]) + b[2:]
        elif r[0] == "1,3,4,6,7":
            r = (r[0], r[1]) + a[2:]
        fixed.append(r)
    return fixed


def test_zone_sizes():
    # z_i = 10, 40, 80, 90, 112, 240, 320 (Table I single-zone rows); total 892 (sc(5)-1..7 row)
    sizes = [len(oracle.zone_offsets(z)) for z in range(1, 8)]
    assert sizes == [10, 40, 80, 90, 112, 240, 320]
    assert len(oracle.mask_offsets(127)) == 892


def test_zone_vectors_by_hand():
    # zone 1 is the 10 unit vectors; zone 4 is 2e_k (10) plus (+-1,+-1,+-1,+-1,0) arrangements (80)
    z1 = {tuple(v) for v in oracle.zone_offsets(1)}
    assert z1 == {tuple(s * np.eye(5, dtype=int)[k]) for k in range(5) for s in (1, -1)}
    z4 = oracle.zone_offsets(4)
    assert sum(1 for v in z4 if max(abs(v)) == 2) == 10
    assert sum(1 for v in z4 if sorted(abs(v)) == [0, 1, 1, 1, 1]) == 80
    # zones 6 and 7: every vector has a +-2 component; zones 1-3 never do
    for z in (6, 7):
        assert all(max(abs(v)) == 2 for v in oracle.zone_offsets(z))
    for z in (1, 2, 3):
        assert all(max(abs(v)) == 1 for v in oracle.zone_offsets(z))
    # every zone is symmetric under v -> -v
    for z in range(1, 8):
        vs = {tuple(v) for v in oracle.zone_offsets(z)}
        assert vs == {tuple(-np.array(v)) for v in vs}


def test_table1_z_zeta_all_127():
    rows = corrected_table1()
    assert len(rows) == 127
    assert sorted(r[1] for r in rows) == list(range(1, 128))
    for label, mask, z, zeta, _ in rows:
        zz, zt = oracle.mask_z_zeta(mask)
        assert zz == z, label
        assert abs(zt - zeta) < 1e-3, (label, zt, zeta)


def test_table1_misprint_is_exactly_the_swap():
    raw = {r[0]: r for r in load_table1()}
    assert oracle.mask_z_zeta(raw["1,3,4,5,7"][1])[0] == 612 != raw["1,3,4,5,7"][2]
    assert oracle.mask_z_zeta(raw["1,3,4,6,7"][1])[0] == 740 != raw["1,3,4,6,7"][2]
    bad = [r[0] for r in load_table1() if oracle.mask_z_zeta(r[1])[0] != r[2]]
    assert sorted(bad) == ["1,3,4,5,7", "1,3,4,6,7"]


def test_table1_pc_never_increases_with_added_zones():
    # with the swap undone, a superset neighborhood never has a larger printed p_c
    rows = corrected_table1()
    pc = {r[1]: r[4] for r in rows}
    for a in range(1, 128):
        for b in range(1, 128):
            if a != b and (a & b) == a:
                assert pc[b] <= pc[a], (a, b)


def test_zeta_single_zone_closed_form():
    for z in range(1, 8):
        n = len(oracle.zone_offsets(z))
        assert math.isclose(oracle.mask_z_zeta(1 << (z - 1))[1], n * math.sqrt(z))


def test_workload_table1_matches_golden():
    """The p grid of the P_max workload is centred on the same (corrected) Table I p_c."""
    from paper_2607_18991_b300 import workloads
    assert {m: pc for (_, m, _, _, pc) in corrected_table1()} == workloads.TABLE1_PC
