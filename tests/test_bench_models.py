"""The benchmark's byte, FLOP and operation models and its clock-sample
parsing, checked on the CPU against hand counts (the roofline fractions in
the bench line are only as good as these)."""
import bench


def test_csr_spmv_bytes_match_the_closed_form():
    # (sv + 4) nnz + 4 (m + 1) + 2 sv m with sv = 8: 5.797 GB at N = 256
    n = 256
    m, nnz = (n + 1) ** 3, (3 * n + 1) ** 3
    b = bench.spmv_bytes("csr", m, (m + 31) // 32, nnz, nnz)
    assert b == 12 * nnz + 4 * (m + 1) + 16 * m
    assert abs(b / 1e9 - 5.7966) < 1e-4


def test_bcrs3_step_model_counts_indices_values_and_vectors():
    m, ns, slots = 1000, 32, 400
    byts, fma, mat = bench.cg_iteration_model("bcrs3", m, ns, slots, 0)
    assert mat == slots * (4 + 3 * 8) + 8 * (ns + 1)
    assert byts == mat + 80 * m          # w=Ap 16 B, r update 24 B, x and p update 40 B per row
    assert fma == 3 * slots + 5 * m      # one FMA per stored value + p.w, r, r.r, x, p


def test_mixed_model_counts_low_and_high_precision_passes():
    m, ns, slots = 1000, 32, 400
    ptrs = 8 * (ns + 1)
    # inner FP32 step: 4 B index + 3 values per slot; vectors in FP32: w = Ap
    # (p, w: 8 B), r and xs update (xs, r, p, w read, xs, r written: 24 B),
    # p update (p, r read, p written: 12 B)
    inner = {"f32": slots * (4 + 3 * 4) + ptrs + 44 * m, "bf16": slots * (4 + 3 * 2) + ptrs + 44 * m}
    # refinement: the FP64 matrix (28 B per slot) + x += xs (24 B) + r = b - A x (20 B)
    hi = slots * 28 + ptrs + 44 * m
    for value in ("f32", "bf16"):
        assert bench.mixed_bytes_model(m, ns, slots, value, 0, 0) == hi   # the initial FP64 residual
        assert bench.mixed_bytes_model(m, ns, slots, value, 7, 2) == 7 * inner[value] + 3 * hi
    # per row at the N = 256 shape (about nine slots per row): 134 B (BF16) and 188 B (FP32)
    n = 256
    m = (n + 1) ** 3
    per_row = {v: (bench.mixed_bytes_model(m, (m + 31) // 32, 9 * m, v, 1, 0)
                   - bench.mixed_bytes_model(m, (m + 31) // 32, 9 * m, v, 0, 0)) / m for v in ("f32", "bf16")}
    assert abs(per_row["bf16"] - 134.25) < 0.01 and abs(per_row["f32"] - 188.25) < 0.01


def test_matrix_free_operation_model_on_a_tiny_cube():
    # N = 2: 27 nodes, one interior node, 26 boundary nodes
    ops = bench.matrix_free_ops(2)
    assert ops["spmv"] == 9
    assert ops["step"] == 12 * 1 + 3 * 26 + 2 * 27
    assert ops["init"] == 10 * 1 + 2 * 27


def test_clock_samples_are_parsed_into_median_and_reasons():
    c = bench.ClockSampler("0")
    c.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0,
                            "kill": lambda self: None})()
    c.lines = ["2070, 2070, 800.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["power_w_max"] == 1390.0


def test_bench_lambda_min_is_the_oracle_spectrum():
    """The bench's forward-error bars use the smallest eigenvalue of the cube's
    Dirichlet system in closed form; it is the oracle's (pinned against dense
    eigenvalues in test_oracle_spectrum.py) for every size."""
    import bench
    import oracle
    for n in list(range(1, 41)) + [96, 128, 256, 400]:
        lo, _ = oracle.dirichlet_extreme_eigenvalues(n, n, n)
        assert abs(bench.lambda_min_cube(n) - lo) <= 1e-12 * lo, n


def test_vbcrs_byte_model_counts_the_paper_arrays():
    """The bench's byte model of the paper's BCRS SpMV: the CRS values, jas and
    offsets per segment (nns = n (3n - 2)^2 on a cube: one segment per row and
    y/z neighbour line, lengths 2 or 3), the segment row pointer, x and y --
    here checked against the oracle's own arrays on a small mesh."""
    import bench
    import oracle
    n = 6
    s = oracle.build_system(n, n, n)
    ptr, jas, off = oracle.csr_to_bcrs(s["row_ptr"], s["cols"])
    nn = n + 1
    assert jas.size == nn * (3 * nn - 2) ** 2
    m, nnz = ptr.size - 1, s["cols"].size
    want = s["vals"].nbytes + jas.nbytes + off.nbytes + ptr.nbytes + 2 * 8 * m
    assert bench.spmv_bytes("vbcrs", m, (m + 31) // 32, jas.size, nnz) == want


def test_reference_arm_times_at_least_40_oracle_iterations(capsys):
    """--impl reference splits at least 40 timed oracle iterations over the timed
    steps (the cpu_baseline leg's sample), on a tiny mesh here."""
    import json
    import sys
    for steps, per_step in ((2, 20), (3, 14), (50, 2)):
        argv = sys.argv
        sys.argv = ["bench.py", "--impl", "reference", "--n", "4", "--steps", str(steps), "--warmup", "0"]
        try:
            bench.main()
        finally:
            sys.argv = argv
        line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
        assert line["impl"] == "reference" and line["gpu_launches"] == 0
        assert f"one oracle call of {per_step} CG iterations" in line["cpu_baseline"]["sample"]
        assert steps * per_step >= 40
