"""Storage precision against the FP64 oracle on a crop of the 8192^2 MIPS
workload: the noise and the initial state are keyed by global site
coordinates, so a 256^2 periodic lattice with the same seed starts from the
top-left crop of the large lattice's initial field.  1000 steps per run.

Asserted: the stated tolerances in the relaxing literal preset (FP32 1e-5,
FP16 storage 2e-3; BF16 storage is held to 2e-3 too and fails it, an expected
failure), and the unstable-regime rule for FP32 in the rescaled preset.  The table (errors and mass drift per storage) is printed with -s.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from lbmtest import errors, gpu_run, oracle_run, split_preset

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("preset", ["MIPS_PAPER_LITERAL", "MIPS_RHO1"])
def test_precision_table(preset, capsys):
    n, steps, seed = 256, 1000, W.seed(3)
    model, d = split_preset(preset)
    spec = W.INIT_CONFIG1
    ref = oracle_run(model, d, n, n, steps, seed, spec)
    m_ref0 = O.observables(O.init(n, n, seed, **spec, prm=O.params(**d)))["mass"]
    rows = []
    res = {}
    for storage in ("f32", "f16s", "bf16s"):
        got = gpu_run(model, d, n, n, steps, seed, spec, storage=storage)
        e_rho, e_u = errors(got, ref)
        drift = (O.observables(np.ascontiguousarray(got))["mass"] - m_ref0) / m_ref0
        res[storage] = (e_rho, e_u)
        rows.append(f"| {preset} | {storage} | {e_rho:.2e} | {e_u:.2e} | {drift:+.2e} |")
    with capsys.disabled():
        print("\n| preset | storage | e_rho | e_u | mass drift |\n|---|---|---|---|---|\n" + "\n".join(rows))
    if preset == "MIPS_PAPER_LITERAL":
        assert max(res["f32"]) <= 1e-5
        assert max(res["f16s"]) <= 2e-3
    else:
        f32 = oracle_run(model, d, n, n, steps, seed, spec, bits=32).astype(np.float64)
        ei = errors(f32, ref)
        with capsys.disabled():
            print(f"| {preset} | FP32 oracle (intrinsic) | {ei[0]:.2e} | {ei[1]:.2e} | - |")
        assert res["f32"][0] <= 4 * ei[0] + 1e-6 and res["f32"][1] <= 4 * ei[1] + 1e-6


@pytest.mark.xfail(strict=True, reason="BF16 shifted storage misses the 2e-3 bound here: e_u = 2.37e-3 measured "
                                       "(8 significand bits on populations whose deviations are the noise itself)")
def test_precision_table_bf16_literal_bound():
    """The stated 2e-3 bound for BF16 storage on the literal preset's 256^2 crop."""
    n, steps, seed = 256, 1000, W.seed(3)
    model, d = split_preset("MIPS_PAPER_LITERAL")
    ref = oracle_run(model, d, n, n, steps, seed, W.INIT_CONFIG1, threads=0)
    got = gpu_run(model, d, n, n, steps, seed, W.INIT_CONFIG1, storage="bf16s")
    assert max(errors(got, ref)) <= 2e-3
