"""The trained warm start against the plain solver (cold start), both to the
same stop rule (rel-x < 1e-5): on unseen 512 x 512 problems the warm start
converges in fewer iterations on average, and its solution has the same
ISNR within 0.05 dB (the stop rule, not the start, decides the result)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.init()
    import paper_1210_2687_gb300.warmstart as mod
    return mod


def test_trained_warm_start_saves_iterations_at_equal_isnr(ws):
    params, scales, meta = ws.load()
    assert params.size == 57252 and meta["lam"] == ws.LAM
    # seeds far from the training and the stored evaluation draws
    probs = [ws.eval_problem(30_000_000 + i) for i in range(8)]
    r = ws.evaluate(params, scales, probs=probs)
    assert r["cold_converged"] == r["warm_converged"] == 8
    assert r["warm_iters_mean"] < r["cold_iters_mean"], r
    assert r["isnr_diff_db_max_abs"] <= 0.05, r
    assert r["prediction_rel_err"]["x"] < 0.15, r
