"""The algorithmic work per element that bench.py divides by measured times
(the roofline's numerators), checked against a line-by-line count of the
plain sum-factorized apply (Section 4.1) and against the per-DOF figures of
the hot-path table (SEM-NI 160 flop/DOF, SEM 277 flop/DOF, FP64 125 B/DOF and
FP32 + bf16 metric 35 B/DOF at p = 4, map excluded)."""
import bench


def _count_flops(p, quad):
    """The 1-D sweeps counted line by line (n outputs of n multiply-adds per
    line, n^2 lines per sweep; SEM-NI 3 gradient and 3 transposed sweeps, SEM
    6 more for the interpolations to and from the Gauss points), plus the
    quadrature-point stage: the 3x3 symmetric product 18, the mass term 2 and
    the sum of the three transposed sweeps 2, 22 flops a point."""
    n = p + 1
    line = 2 * n * n                   # n outputs, n multiply-adds each
    lines_per_sweep = n * n
    sweeps = 6 if quad == "LGL" else 12  # gradient + transpose; SEM adds 6 interpolations
    return sweeps * lines_per_sweep * line + 22 * n ** 3


def test_flops_per_element_match_line_count():
    for p in range(1, 7):
        for quad in ("LGL", "LG"):
            assert bench.apply_flops_per_element(p, quad) == _count_flops(p, quad)


def test_per_dof_figures_at_p4():
    p, n = 4, 5
    dofs = p ** 3  # nodes per element in the interior of a large mesh
    assert round(bench.apply_flops_per_element(p, "LGL") / dofs) == 160
    assert round(bench.apply_flops_per_element(p, "LG") / dofs) == 277
    assert round((bench.apply_bytes_per_element(p) - 4 * n ** 3) / dofs) == 125
    assert round((bench.apply_bytes_per_element_fp32(p, "bf16") - 4 * n ** 3) / dofs) == 35


def test_bytes_per_element_components():
    for p in range(1, 7):
        n = p + 1
        # FP64: 7 doubles per point, int32 map, u read + y written (8 + 8) per node
        assert bench.apply_bytes_per_element(p) == 7 * 8 * n ** 3 + 4 * n ** 3 + 16 * p ** 3
        # FP32 arithmetic with the bf16 metric: 7 x 2 B per point, map, 4 + 4 B per node
        assert bench.apply_bytes_per_element_fp32(p, "bf16") == 7 * 2 * n ** 3 + 4 * n ** 3 + 8 * p ** 3


def test_kernel_source_hash_ignores_comments_only():
    """The source hash that keys the ncu traffic figures changes with the code
    and not with comments or blank lines."""
    code = "int f(int a) {\n  return a + 1;\n}\n"
    commented = "// adds one\nint f(int a) {  // the argument\n\n  return a + 1;  /* the sum */\n}\n"
    changed = "int f(int a) {\n  return a + 2;\n}\n"
    assert bench._code_only(code) == bench._code_only(commented)
    assert bench._code_only(code) != bench._code_only(changed)
    assert len(bench.kernel_source_hash("apply")) == 16
