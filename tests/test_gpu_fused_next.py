"""gs_project_bwd_adam_next: the fused optimizer pass that also projects the
updated parameters into the next training step's view. It must agree with
gs_project_bwd_adam followed by gs_project of the updated parameters, in every
SH storage form, up to FP32 rounding where the two kernels' compiled arithmetic
differs; and a training step that takes the next view must agree with one
that projects on its own."""
import numpy as np
import pytest
import torch

from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300 import scenes
from paper_2412_13547_b300.pipeline import Rasterizer, TrainStep

import gpu_util as U

pytestmark = pytest.mark.gpu


def _scene(deg):
    if deg == 0:
        s, cam, _ = scenes.workload_small()
        return U.params_np(s), cam
    s = scenes.small_scene(3000, index=11, sh_degree=3, log_scale_mean=-2.6)
    s.sh[:, 1:, :] = np.random.default_rng(5).normal(0, 0.1, s.sh[:, 1:, :].shape)
    return U.params_np(s), scenes.look_at(scenes.orbit_eye(3.0, 60.0, 25.0), width=160, height=120)


def _outputs(n):
    return dict(splats=torch.zeros(n, R.SPLAT_FLOATS, device=U.DEV),
                radii=torch.zeros(n, dtype=torch.int32, device=U.DEV),
                rects=torch.zeros(n, 4, dtype=torch.int32, device=U.DEV),
                tiles_touched=torch.zeros(n, dtype=torch.int32, device=U.DEV),
                depth_keys=torch.zeros(n, dtype=torch.int32, device=U.DEV))


@pytest.mark.parametrize("sh_dtype,master,deg", [(torch.float32, False, 3), (torch.bfloat16, False, 3),
                                                (torch.float16, False, 3), (torch.bfloat16, True, 3),
                                                (torch.float32, False, 0)],
                         ids=["fp32", "bf16", "fp16", "fp32_master_bf16", "fp32_sh0"])
def test_fused_pass_projects_the_next_view(sh_dtype, master, deg):
    """Two steps in a row (the second from the projection the first one wrote):
    * the projection it writes is gs_project of the parameters it leaves: rects,
      radii, tile counts, depth keys, centres, opacities and colours bit for bit;
      the conic up to its FP32 rounding (the compiler contracts its products
      differently in the two kernels), within 1e-4 of its scale;
    * parameters, moments and statistics are gs_project_bwd_adam's up to the FP32
      rounding of the gradient arithmetic (as between the fused and unfused
      optimizer paths): a few elements one rounding apart, which Adam keeps within
      2 lr."""
    p32, cam = _scene(deg)
    d0, d1 = R.Dilation(2, 1, 0, bin_shift=1), R.Dilation(2, 0, 1, bin_shift=1)
    out, rast, p, (img, tf, last) = U.run_forward(p32, cam, d0, sh_dtype=sh_dtype, master=master)
    dl = torch.tensor(np.random.default_rng(4).standard_normal(img.shape) * 1e-3, dtype=torch.float32,
                      device=U.DEV)
    rast.render_bwd(cam, d0, (0.0, 0.0, 0.0), tf, last, dl)
    lrs = [1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3]
    n = p.n
    sets = []
    for _ in range(2):
        ps = [t.clone() for t in p.tensors()]
        sets.append(dict(p=ps, m=[torch.zeros_like(t, dtype=torch.float32) for t in ps],
                         v=[torch.zeros_like(t, dtype=torch.float32) for t in ps],
                         shadow=p.sh_store.clone() if master else None,
                         stats=[torch.zeros(n, device=U.DEV), torch.zeros(n, device=U.DEV),
                                torch.zeros(n, dtype=torch.int32, device=U.DEV)],
                         tiles=rast.tiles_touched.clone(), out=_outputs(n)))
    a, b = sets
    for step in (1, 2):
        store_a = a["shadow"] if a["shadow"] is not None else a["p"][4]
        store_b = b["shadow"] if b["shadow"] is not None else b["p"][4]
        R.gs_project_bwd_adam(a["p"], a["m"], a["v"], lrs, 0.9, 0.999, 1e-15, step, store_a, cam, d0,
                              a["tiles"], rast.grad2d, sh_shadow=a["shadow"], pos_acc=a["stats"][0],
                              col_acc=a["stats"][1], count=a["stats"][2], sr_seed=9)
        # the fused form writes its tile counts over the ones it reads
        b["out"]["tiles_touched"] = b["tiles"]
        R.gs_project_bwd_adam_next(b["p"], b["m"], b["v"], lrs, 0.9, 0.999, 1e-15, step, store_b, cam, d0,
                                   b["tiles"], rast.grad2d, R.View(cam, d1, **b["out"]), sh_shadow=b["shadow"],
                                   pos_acc=b["stats"][0], col_acc=b["stats"][1], count=b["stats"][2], sr_seed=9)
        ref = _outputs(n)
        R.gs_project(*b["p"][:4], store_b, cam, d1, ref["splats"], ref["radii"], ref["rects"],
                     ref["tiles_touched"], depth_keys=ref["depth_keys"])
        torch.cuda.synchronize()
        for k in ("radii", "rects", "tiles_touched", "depth_keys"):
            assert torch.equal(ref[k], b["out"][k]), (step, k)
        s_ref, s_b = ref["splats"], b["out"]["splats"]
        exact = [c for c in range(R.SPLAT_FLOATS) if c not in (2, 3, 4)]
        assert torch.equal(s_ref[:, exact], s_b[:, exact]), step
        scale = s_ref[:, 2].abs() + s_ref[:, 4].abs() + 1e-30
        assert ((s_ref[:, 2:5] - s_b[:, 2:5]).abs().max(1).values / scale).max().item() < 1e-4
        assert int((b["tiles"] > 0).sum().item()) > 0
        for x, y, lr in zip(a["p"], b["p"], lrs):
            diff = (x.float() - y.float()).abs()
            assert diff.max().item() <= 2.0 * lr * 1.01 + 1e-6
            assert (diff > 1e-6 * (1.0 + y.float().abs())).float().mean().item() < 0.01
        for x, y in zip(a["stats"], b["stats"]):
            assert torch.allclose(x.float(), y.float(), rtol=1e-5, atol=1e-9)
        # the next step of each path starts from its own tile counts
        a["tiles"] = (b["tiles"] > 0).to(torch.int32) * b["tiles"]


def test_train_step_with_the_next_view_equals_projecting_each_step():
    """TrainStep(..., next_view=...) skips the next step's projection: the losses, images
    and parameters of steps that project on their own, up to what float atomics in another
    order change (the blend backward's; Adam can turn the sign of a near-zero gradient into a
    full +-lr step, so a few elements may differ by up to 2 lr)."""
    p32, cam = _scene(3)
    tgt = torch.tensor(scenes.quantize_u8(scenes.target_image(cam.width, cam.height, 11)), device=U.DEV)
    dils = [R.Dilation(2, ox, oy, bin_shift=1) for oy in range(2) for ox in range(2)]
    runs = []
    for use_next in (False, True):
        p = U.gpu_params(p32)
        rast = Rasterizer(p.n, capacity=1 << 18, max_grid=R.gs_bin_grid(cam, R.Dilation(2, 0, 0, bin_shift=1)))
        w, h, _, _ = R.gs_grid(cam, dils[0])
        st = TrainStep(p, rast, max_pixels=w * h)
        losses, proj = [], []
        for i in range(6):
            nxt = (cam, dils[(i + 1) % 4]) if use_next else None
            losses.append(float(st(cam, dils[i % 4], tgt, next_view=nxt).item()))
            proj.append(st.projected)
        torch.cuda.synchronize()
        runs.append((losses, [t.clone() for t in p.tensors()], st.img.clone(), proj))
    np.testing.assert_allclose(runs[0][0], runs[1][0], rtol=1e-4)
    lrs = [st.adam.lr_means, st.adam.lr_log_scales, st.adam.lr_quats, st.adam.lr_opacity, st.adam.lr_sh]
    for x, y, lr in zip(runs[0][1], runs[1][1], lrs):
        diff = (x - y).abs()
        assert diff.max().item() <= 2.0 * lr * 1.01 + 1e-6
        assert (diff > 1e-6 * (1.0 + y.abs())).float().mean().item() < 0.01
    assert (runs[0][2] - runs[1][2]).abs().max().item() < 1e-2
    assert runs[0][3] == [True] * 6 and runs[1][3] == [True] + [False] * 5


def test_reallocated_parameters_or_another_view_project_again():
    """The projection an optimizer pass carries to the next step is used only for the view it was
    made for and the tensors it was made from: another view, or parameters reallocated between
    the steps (as densification does), make the step project on its own."""
    p32, cam = _scene(0)
    tgt = torch.tensor(scenes.quantize_u8(scenes.target_image(cam.width, cam.height, 3)), device=U.DEV)
    d0, d1 = R.Dilation(2, 0, 0, bin_shift=1), R.Dilation(2, 1, 0, bin_shift=1)
    p = U.gpu_params(p32)
    rast = Rasterizer(p.n, capacity=1 << 18, max_grid=R.gs_bin_grid(cam, d0))
    w, h, _, _ = R.gs_grid(cam, d0)
    st = TrainStep(p, rast, max_pixels=w * h)
    st(cam, d0, tgt, next_view=(cam, d1))
    st(cam, d0, tgt, next_view=(cam, d1))  # not the view the last pass projected into
    assert st.projected
    st(cam, d1, tgt, next_view=(cam, d0))  # the carried projection
    assert not st.projected
    p.means = p.means.clone()  # reallocated between the steps
    st(cam, d0, tgt)
    assert st.projected
    torch.cuda.synchronize()
