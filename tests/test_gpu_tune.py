"""The plan autotuner: on three seeded shapes (a 2D quadratic one-shot transfer, a 3D
quadratic operator with 8 fields, a 2D linear operator with dense neighbourhoods), the tuned
table's plans are never slower than the plan rules' (timed again after tuning, with a 10%
allowance for timing noise), and they give the same results within the mixed tolerance."""
import numpy as np
import pytest

from tests._helpers import TOL_MIXED, need_gpu, normwise_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    need_gpu()
    from paper_2510_18838_gb300 import build, pcms, tune
    build.build()
    return pcms, tune


def test_tuned_plans_are_never_slower_and_agree(env):
    import torch
    pcms, tune = env
    shapes = [tune.Shape(2, 2, "oneshot", 40.0, 150_000, 1, seed=11),
              tune.Shape(3, 2, "map", 57.0, 150_000, 8, seed=12),
              tune.Shape(2, 1, "map", 150.0, 150_000, 4, seed=13)]
    try:
        table = tune.tune(shapes, reps=3, apply_fields=(8,))
        entries = table["entries"]
        assert len(table["measurements"]) == len(shapes) + 1
        for sh in shapes:
            prob = tune._problem(sh, torch.device("cuda", 0))
            pcms.tune_set([])
            t_rule = tune.time_call(lambda: tune._call(sh, prob), 5)
            out_rule = tune._call(sh, prob).cpu().numpy()
            pcms.tune_set(entries)
            t_tuned = tune.time_call(lambda: tune._call(sh, prob), 5)
            out_tuned = tune._call(sh, prob).cpu().numpy()
            assert t_tuned <= 1.10 * t_rule + 0.05, (sh, t_tuned, t_rule, entries)
            ok = np.isfinite(out_rule).all(axis=0)
            assert np.array_equal(np.isfinite(out_tuned).all(axis=0), ok)
            assert normwise_err(out_tuned, out_rule, ok) <= TOL_MIXED
        got = pcms.tune_get()
        assert len(got) == len(entries)
    finally:
        pcms.tune_set([])
