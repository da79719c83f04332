"""End-to-end fit on a small scene: both forms (plain full-resolution FP32 one
view per step, and dilated + BF16 + batched) lower the held-out error, the
densification rounds grow the Gaussians within the budget, and the step
kernels see no pair-capacity overflow."""
import numpy as np
import pytest
import torch

from paper_2412_13547_b300 import scenes
from paper_2412_13547_b300.densify import DensifyConfig
from paper_2412_13547_b300.fit import Fit, FitConfig, psnr, render_views, time_to_psnr
from paper_2412_13547_b300.pipeline import AdamConfig, GaussianParams

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def problem():
    gt, init, train, held = scenes.fit_workload(n_gt=30000, n_init=3000, n_train=24, n_eval=3, width=320,
                                                height=192)
    gp = GaussianParams.from_arrays(gt.as_dict(), DEV)
    train_t = render_views(gp, train)
    eval_t = render_views(gp, held)
    assert psnr(gp, held, eval_t) > 90.0  # the ground truth reproduces its own renders
    return init, train, train_t, held, eval_t


@pytest.mark.parametrize("form", ["plain", "turbo"])
def test_fit_improves_and_densifies(problem, form):
    init, train, train_t, held, eval_t = problem
    cfg = FitConfig(form=form, views=960, views_per_step=4, budget=9000, densify_from=160, densify_until=800,
                    densify_every=160, eval_every=480, adam=AdamConfig(lr_means=2e-4, lr_sh=5e-3),
                    densify=DensifyConfig(tau_pos=1e-7, split_scale=0.03, min_opacity=0.005))
    fit = Fit(cfg, init, train, train_t, held, eval_t)
    hist = fit.run()
    assert hist[-1]["psnr"] > hist[0]["psnr"] + 1.0, hist
    assert len(fit.rounds) >= 3
    assert hist[-1]["n"] > 3000
    assert max(h["n"] for h in hist) <= int(1.5 * 9000)
    for r in fit.rounds:
        assert r["n_grown"] - r["n_before"] <= r["max_new"]
    assert all(np.isfinite(h["psnr"]) for h in hist)
    assert time_to_psnr(hist, hist[0]["psnr"]) == 0.0
