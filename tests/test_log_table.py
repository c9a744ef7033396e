"""The table-driven logarithm of the FP64 direct sum (Tang's method: 128
interval centres c = 1 + (2k + 1)/256, log(1 + t) to t^6), checked as
mathematics on the CPU: the same steps in numpy float64 against numpy's log,
over values spanning every exponent the 2D kernel meets and every interval
of the table.  The device code itself is checked against the oracle's
direct sum by the GPU parity suite."""
import numpy as np


def _log_tab(x):
    u = x.view(np.uint64)
    ef = ((u >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    k = ((u >> np.uint64(45)) & np.uint64(127)).astype(np.int64)
    m = ((u & np.uint64(0x000FFFFFFFFFFFFF)) | np.uint64(0x3FF0000000000000)).view(np.float64)
    c = 1.0 + (2 * k + 1) * (1.0 / 256.0)
    t = (m - c) * (1.0 / c)
    q = t * (-1.0 / 6.0) + 1.0 / 5.0
    q = t * q - 0.25
    q = t * q + 1.0 / 3.0
    q = t * q - 0.5
    l1p = (t * t) * q + t
    return (ef - 1023) * 0.69314718055994530942 + (np.log(c) + l1p)


def test_table_log_error_bound():
    rng = np.random.default_rng(3)
    # every table interval at unit scale, then squared distances 1e-12..1e4
    x = np.concatenate([1.0 + (np.arange(128 * 64) + 0.5) / (128 * 64),
                        10.0 ** rng.uniform(-12, 4, 200000)])
    ref = np.log(x)
    err = np.abs(_log_tab(x) - ref)
    # a few units of 2^-53 times max(1, |log x|) (numpy's own log and the
    # unfused steps here add their roundings); a series one term shorter
    # would leave up to 5.3 units at the interval edges
    assert (err <= 4 * 2.0 ** -53 * np.maximum(1.0, np.abs(ref))).all(), err.max()


def test_table_log_exact_at_powers_of_two():
    e = np.arange(-40, 14)
    x = np.ldexp(1.0, e)
    assert np.allclose(_log_tab(x), e * np.log(2.0), rtol=0, atol=4e-16 * 40)
