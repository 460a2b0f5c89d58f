"""Host-side pieces of bench.py: the algorithmic byte model (per RK4 step, per
kernel kind) against the sizes written out by hand for the benchmark element
(tetrahedron, p = 3, Euler, FP32), and the workload labels."""
import pytest

bench = pytest.importorskip("bench")

TET3 = {"nsol": 20, "nfe": 40, "nfiu": 10, "nfaces": 4, "ndim": 3}


def test_record_path_bytes_per_element():
    s, V = 4, 5
    b = bench.algorithmic_bytes(TET3, 1, V, s, record=True, viscous=False)
    # interpolation: read U (20 x 5), write 40 + 10 point states -> 70 x 5 x 4 B, four per step
    assert b["interp_ext"] == 4 * 1400
    # flux per stage: own + partner external states (2 x 40 x 5 x 4 = 1,600), internal
    # states (200), metric 26 values (104), permutation 40 B, partner offsets 16 B;
    # stage updates 13 state volumes of 400 B per step
    assert b["residual"] == 4 * (1600 + 200 + 104 + 40 + 16) + 13 * 400


def test_fused_rk_bytes_per_element():
    s, V = 4, 5
    unf = bench.algorithmic_bytes(TET3, 1, V, s, record=True, viscous=False)
    fus = bench.algorithmic_bytes(TET3, 1, V, s, record=True, viscous=False, fused=True)
    # one interpolation per step instead of four
    assert fus["interp_ext"] == unf["interp_ext"] / 4
    # stages 1-3 write the next records (50 point states) instead of the stage state
    assert fus["residual"] == unf["residual"] - 3 * 400 + 3 * 50 * V * s
    total_unf = sum(unf.values())
    total_fus = sum(fus.values())
    assert total_fus < total_unf


def test_workload_labels():
    assert bench.workload_label("euler") == "euler3d_tet_p3_82944_rk4"
    assert bench.workload_label("tgv") == "tgv_ns_tet_p4_663552_rk4"
    assert bench.workload_label("mixed").startswith("mixed_euler_") and bench.workload_label("mixed").endswith("_rk4")


def test_solution_point_counts_match_the_paper_table():
    """bench.N_SOL (used to project the reference arm's step time) against the
    counts of App. A's table in tests/golden/point_counts.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "point_counts.txt")
    seen = 0
    for line in open(path):
        parts = line.split()
        if not parts or parts[0].startswith("#") or parts[0] not in bench.N_SOL:
            continue
        shape, p, nsol = parts[0], int(parts[1]), int(parts[2])
        assert bench.N_SOL[shape](p) == nsol, (shape, p)
        seen += 1
    assert seen >= 20


def test_clock_sample_parsing():
    out = "\n".join([
        "0, 2070, 2070, 812.45, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1390.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1965, 2070, 1398.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage"])
    c = bench.ClockSampler.parse(out)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    empty = bench.ClockSampler.parse("")
    assert empty["sm_mhz"] is None and empty["samples"] == 0


def test_full_size_dof_counts():
    """The reference arm's projection uses element counts without building the
    mesh: the counts of the workloads' stated sizes."""
    assert bench.full_ndof("euler") == 82944 * 20 * 5
    assert bench.full_ndof("tgv") == 663552 * 35 * 5
    # mixed: hexahedra / x-prisms p1, tets / z-prisms p2, hexahedra / x-prisms p3, tets / z-prisms p4
    want = (40 * 40 * (100 * 8 + 44 * 2 * 6) + 32 * 32 * (16 * 6 * 10 + 10 * 2 * 18)
            + 24 * 24 * (45 * 64 + 21 * 2 * 40) + 16 * 16 * (11 * 6 * 35 + 6 * 2 * 75)) * 5
    assert bench.full_ndof("mixed") == want == 34624000


def test_byte_models_per_element():
    """Residual bytes s V (3 N_s + 2 N_fe) + geometry + connectivity for the
    degree-3 tetrahedron (FP32, Euler): 4 * 5 * (60 + 80) + (1 + 9 + 16) * 4 + 32."""
    assert bench.residual_bytes(TET3, 5, 4, False) == 2800 + 104 + 32
    g = bench.generated_bytes(TET3, 5, 4)
    vol, rec, side = 400, 800, 104 + 160
    assert g["interp_ext"] == vol + rec
    assert g["residual"] == 4 * (vol + rec + side) + 13 * vol + 3 * rec
