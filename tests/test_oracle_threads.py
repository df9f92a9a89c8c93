"""The threaded oracle build (OpenMP over rows) computes exactly what the
single-thread oracle computes: each site's arithmetic is the same sequence in
the same order, only the rows are shared out among host threads."""
import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.mark.parametrize("name", ["MIPS_RHO1", "CIL_RHO1", "PASSIVE"])
@pytest.mark.parametrize("threads", [2, 5])
def test_threaded_run_is_bitwise_single_thread(name, threads):
    d = W.preset(name)
    model = d.pop("model")
    p = O.params(**d)
    f = O.init(48, 38, 99, **W.INIT_CONFIG2, prm=p)
    a = O.run(f, model, p, 99, 3, 12)
    b = O.run(f, model, p, 99, 3, 12, threads=threads)
    np.testing.assert_array_equal(a, b)
    assert O.threads_in_use(threads) == threads


@pytest.mark.parametrize("name", ["MIPS_RHO1", "CIL_RHO1"])
def test_threaded_run7_and_window_are_bitwise_single_thread(name):
    d = W.preset(name)
    model = d.pop("model")
    p = O.params(**d)
    f = O.init7(30, 22, 5, **W.INIT_CONFIG2, prm=p)
    np.testing.assert_array_equal(O.run7(f, model, p, 5, 0, 10), O.run7(f, model, p, 5, 0, 10, threads=3))
    win = (100, 40, 512, 512)
    g = O.init(36, 20, 5, **W.INIT_CONFIG1, prm=p, window=win)
    np.testing.assert_array_equal(O.run(g, model, p, 5, 0, 6, window=win),
                                  O.run(g, model, p, 5, 0, 6, window=win, threads=0))


def test_threaded_oracle_is_fp64_only():
    p = O.params()
    with pytest.raises(ValueError):
        O.run(np.zeros((9, 4, 4), np.float32), "passive", p, 0, 0, 1, bits=32, threads=2)
