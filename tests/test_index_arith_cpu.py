"""Index arithmetic that the CUDA kernels take in FP32 instead of an integer division, checked exhaustively
over the ranges the kernels can see (numpy's float32 add, multiply and divide round to nearest, as the GPU's
do with the library's flags):
- the PCG kernel's first product splits its work items t into (block row k, input j) with
  k = (int)((t + 0.5) * (1 / nu)), for t < N nu, N <= SSPCG_MAX_N = 4096, nu <= 28;
- the padding kernel finds the row of a 16-byte piece v of padded rows of q = width / 4 pieces with
  r = (int)((v + 0.5) * (1 / q)), for v < 4096 * 28 rows * q, q <= 7.
Both must equal the integer quotient."""
import numpy as np


def _float_quotient(v, d):
    inv = np.float32(1.0) / np.float32(d)
    return ((v.astype(np.float32) + np.float32(0.5)) * inv).astype(np.int64)


def test_pcg_item_split_is_exact():
    for nu in range(1, 29):
        t = np.arange(4096 * nu, dtype=np.int64)
        assert np.array_equal(_float_quotient(t, nu), t // nu), nu


def test_padding_piece_row_is_exact():
    for q in range(1, 8):
        v = np.arange(4096 * 28 * q, dtype=np.int64)
        assert np.array_equal(_float_quotient(v, q), v // q), q
