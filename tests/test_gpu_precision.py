"""Tensor-core precision forms (BF16 / FP16 DFT stages, FP32 accumulation)
against the FP64 oracle.

The DFT matrices and the scaled data are rounded to 16 bits, so a single
transform carries a relative error of about 2^-9 (BF16, 8-bit significand)
or 2^-12 (FP16, 11 bits) times a small growth factor; one iteration chains
four transform passes.  Bounds per iteration from an oracle state:
BF16 2e-2, FP16 3e-3 relative L2 (the FP32 engine: 1e-4).  The measured
errors are printed.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

BOUND = {1: 2e-2, 2: 3e-3}


@pytest.fixture(scope="module")
def cp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_05283_gb300 as pkg
    return pkg


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).astype(np.float64)
    b = b.reshape(b.shape[0], -1).astype(np.float64)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("N,Np", [(64, 4), (128, 3), (256, 2), (512, 2), (1024, 1)])
@pytest.mark.parametrize("prec", [1, 2])
def test_tc_er_steps_track_oracle(cp, N, Np, prec):
    d = synth.make_case("tiny", N=N, Np=Np)
    S = (d["proj"].numpy() > 1e-9).astype(np.uint8)  # tight support: ER is contractive
    iters = 5
    cfg = cp.make_config(N, Np, seed=3, hio_iters=0, er_iters=iters, n_ei=3, precision=prec)
    plan = cp.Plan(cfg)
    plan.load_intensities(d["I"], 0, d["thetas"])
    plan.load_support(S)
    errs = plan.iterate(iters, errors=True)
    g = plan.result(cp.RESULT_STATE)
    plan.close()
    run = O.OracleRun.start(O.OracleConfig(N=N, Np=Np, seed=3, hio_iters=0, er_iters=iters, n_ei=3,
                                           beta=float(np.float32(0.9))), d["I"], S).run(iters)
    rel = _rel(g, run.g).max()
    erel = np.max(np.abs(errs - np.array(run.errors)) / np.array(run.errors))
    print(f"N={N} prec={prec}: iterate rel-L2 {rel:.2e} after {iters} ER iterations, "
          f"error-metric rel {erel:.2e}")
    assert rel < BOUND[prec] * iters
    assert erel < BOUND[prec] * iters


def test_tc_precision_rejected_off_warp_engine(cp):
    with pytest.raises(cp.CpraError) as e:
        cp.Plan(cp.make_config(96, 2, precision=1))
    assert e.value.status == cp.ERR_UNSUPPORTED
    with pytest.raises(cp.CpraError) as e:
        cp.Plan(cp.make_config(64, 2, precision=1, engine=cp.ENGINE_TWO_PASS))
    assert e.value.status == cp.ERR_UNSUPPORTED
