"""The bench's byte and flop models (host only): the figures the roofline
objects divide by, checked against counts done by hand for the 512^3 model
insect and against their definitions on small grids."""
import math

import bench


def test_kept_mode_counts():
    # 2/3 rule, kept |m| <= floor(n/3): x keeps 0..170, y and z keep -170..170
    assert bench.spectral_sizes((512, 512, 512)) == (171, 341, 341)
    assert bench.spectral_sizes((96, 96, 192)) == (33, 65, 129)


def test_xpass_bytes_512():
    """6 fields in and 3 out, nz ny rows of Mx complex FP32 values each."""
    kb = bench.kernel_bytes((512, 512, 512), 4)
    row = 171 * 8
    assert kb["xpass_phys"] == 9 * 512 * 512 * row == 3227516928
    # every pass reads and writes each value once: the y inverse turns the
    # six My-row fields into ny-row ones
    A, B = 512 * 341 * row, 512 * 512 * row
    assert kb["yinv"] == 6 * A + 6 * B
    assert kb["zinv_curl"] == 3 * 341 * 341 * row + 6 * A
    # the step runs one of the two x kernels (CUDA-core or tensor-core), same bytes
    assert kb["xpass_tc"] == kb["xpass_phys"]
    assert sum(v for k, v in kb.items() if k != "xpass_tc") == 14094707832


def test_xpass_flops_512():
    """Nine half-length complex FFTs (m = 256: 5 m log2 m = 10 240 flops),
    their mirror steps (14 flops per output) and 15 flops per point, per row."""
    per_row = 9 * (5 * 256 * 8 + 14 * 256) + 15 * 512
    assert per_row == 132096
    assert bench.xpass_flops((512, 512, 512)) == 512 * 512 * per_row
    assert math.isclose(bench.xpass_flops((512, 512, 512)) / 1e9, 34.628, rel_tol=1e-4)
    # the wake terms add six more line transforms per row
    assert bench.xpass_flops((64, 8, 8), wake=True) > bench.xpass_flops((64, 8, 8))


def test_fp32_peak():
    assert math.isclose(bench.FP32_PEAK_TFLOPS, 80.54784)


def test_xpass_tc_flops():
    """Tensor-core flops of the split-BF16 x pass, counted by hand at 512^3:
    32 768 tiles of 8 rows, per line two products of 128 x 32 x 32 (the two
    16-point stages), 2 flops per multiply-add, three piece products (hi+lo)
    or six (hi+mid+lo)."""
    per_line = 2 * 128 * 32 * 32
    assert bench.xpass_tc_flops((512, 512, 512), 2) == 2 * 32768 * 9 * per_line * 3
    assert bench.xpass_tc_flops((512, 512, 512), 3) == 2 * bench.xpass_tc_flops((512, 512, 512), 2)
    # nx = 256: 16-row tiles, a stage of two 128 x 16 x 16 products and one of 128 x 32 x 32
    assert bench.xpass_tc_flops((256, 16, 16), 2) == 2 * 16 * 9 * (2 * 128 * 16 * 16 + 128 * 32 * 32) * 3


def test_kernel_flops_512():
    """FP64 roofline flops: y inverse = 6 fields x nz Mx lines of a 512-point
    FFT (5 m log2 m = 23 040 flops), y forward half of it, the x pass as
    xpass_flops; the step at 512^3 totals about 65 GFLOP (pruned modes)."""
    kf = bench.kernel_flops((512, 512, 512))
    assert kf["yinv"] == 6 * 512 * 171 * 5 * 512 * 9
    assert kf["yfwd"] * 2 == kf["yinv"]
    assert kf["xpass_phys"] == bench.xpass_flops((512, 512, 512)) == kf["xpass_tc"]
    assert kf["zfwd"] == 3 * 341 * 171 * 5 * 512 * 9
    step = sum(v for k, v in kf.items() if k != "xpass_tc")
    assert 6.4e10 < step < 6.6e10
