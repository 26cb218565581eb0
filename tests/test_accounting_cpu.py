"""Operation accounting of the benchmark against the figures the paper prints
(no GPU).  The paper gives no worked outputs, but its operation counts fix
the conventions: Sec. 4 puts the full-array correlation at about one
TFLOP per subband-second, and Table 2 (Sec. 8) gives compute time x rate
for the FIR and FFT, which multiply out to the counts below."""
import math

import bench

S = 195313          # samples per one-second subband (195,312.5 Hz)


def test_xengine_ops_match_one_tflop_per_subband():
    """8 real ops per complex MAC, lower triangle with autocorrelations:
    8 * 1152*1153/2 * 195,313 = 1.038e12, the paper's "about 1 TFLOP per
    subband for the full array" (Sec. 4)."""
    ops = bench.xops(1152, S, 1, 1)
    assert ops == 8 * (1152 * 1153 // 2) * S
    assert abs(ops / 1.04e12 - 1) < 0.01
    # channelising into C channels keeps the count: T spectra x C channels = S samples
    assert bench.xops(1152, S // 64, 64, 1) == 8 * (1152 * 1153 // 2) * (S // 64) * 64
    # A-6 is a quarter: four times fewer baselines
    assert abs(bench.xops(576, S, 1, 1) / ops - 576 * 577 / (1152 * 1153)) < 1e-12


def test_table2_fir_and_fft_rows():
    """Table 2, A-12: FIR 31.1 ms x 0.466 TFLOP/s and FFT 18.6 ms x 0.488 TFLOP/s
    reproduce a 16-tap complex-by-real FIR (4 flop per tap and sample) and a
    256-point FFT at 5 C log2 C flop, to 1.5%; A-6 is half of each."""
    fir = 1152 * S * 16 * 4
    fft = 1152 * (S / 256) * 5 * 256 * math.log2(256)
    assert abs(31.1e-3 * 0.466e12 / fir - 1) < 0.015
    assert abs(18.6e-3 * 0.488e12 / fft - 1) < 0.015
    assert abs(13.2e-3 * 0.547e12 / (fir / 2) - 1) < 0.015
    assert abs(9.18e-3 * 0.493e12 / (fft / 2) - 1) < 0.015
