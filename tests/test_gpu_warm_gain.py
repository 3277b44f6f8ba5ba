"""What the learned warm start gains over the method without it.

The family of the learned-warm-start workload (horizon 15, branching 4 for 4 stages, nx = 20,
nu = 10): the batched NAMA solves the configured 50,000 training draws, the tensor-core network
is trained on their duals (10 epochs, Adam), and 1,000 held-out draws are solved from y0 = 0 and
from the learned start with the phi fallback (a draw whose predicted start has a higher FBE than y0 = 0
starts cold).  Every draw must reach the tolerance both ways, the warm starts must need fewer
NAMA iterations on average than the cold starts, and the fallback must keep every draw's first
FBE at or below its cold value."""
import numpy as np
import pytest
import torch

from paper_2107_01745_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_learned_start_needs_fewer_iterations(cuda_device):
    from paper_2107_01745_b300 import warmstart as WS
    system = W.warm_start_system(4)
    lam = WS.batch_lambda(system)
    data = WS.make_dataset(system, W.WARM_TRAIN_SEED, 50000, lam)
    starter = WS.WarmStarter(system, hidden=256, batch=8192, seed=0)
    fit = starter.fit(data, epochs=10, lr=1e-3)
    del data
    assert np.isfinite(fit["loss"]).all() and fit["loss"][-50:].mean() < 0.5 * fit["loss"][:10].mean()
    ev = WS.EvalSet(W.warm_start_draws(system, W.WARM_EVAL_SEED, 1000, dtype=np.float32), lam)
    r = WS.warm_vs_cold(starter, ev)
    print("learned warm start: cold iters %.3f (max %d), warm iters %.3f (max %d), fallbacks %d, "
          "cold %.1f ms, warm %.1f ms" % (r["cold_iters_mean"], r["cold_iters_max"], r["warm_iters_mean"],
                                           r["warm_iters_max"], r["fallbacks"], r["cold_ms"], r["warm_ms"]))
    assert r["converged"]
    assert r["warm_iters_mean"] < r["cold_iters_mean"]
    # the fallback keeps the start no worse than y0 = 0 in the quantity NAMA decreases
    start, _ = WS.choose_start(ev, r["y0"])
    assert np.all(ev.phi(start) <= ev.phi(None) + 1e-6 * np.maximum(1.0, np.abs(ev.phi(None))))
    ev.close()
