"""Batched views: one launch per stage over several views of uneven
resolution and dilation must give each view the results of the one-view
calls, which the parity tests pin to the FP64 oracle; one view of a batch is
also compared with the oracle directly.

What is deterministic is compared bit for bit (projection, binning, forward
blend, loss gradient); what goes through float atomics in a different order
(backward blend, loss value) or sums views in a different association
(fused backward + Adam) within FP32 rounding.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2412_13547_b300 import raster as R
from paper_2412_13547_b300 import scenes
from paper_2412_13547_b300.pipeline import AdamConfig, BatchTrainStep, GaussianParams, autotune_batch

import gpu_util as U

pytestmark = pytest.mark.gpu

DEV = "cuda"
BG = (0.1, 0.2, 0.3)


def batch_scene(n=30000, tile=16):
    """Four views around a clustered scene with a packed ball: ragged sizes,
    dilations 1..3 with different offsets."""
    s = scenes.cluster_scene(n, index=7, log_scale_mean=-3.6, packed_frac=0.2, packed_radius=0.25)
    spec = [((320, 180), 30.0, 15.0, R.Dilation(1, 0, 0, tile=tile)),
            ((257, 193), 120.0, 40.0, R.Dilation(2, 1, 0, tile=tile)),
            ((400, 224), 210.0, 5.0, R.Dilation(1, 0, 0, tile=tile)),
            ((161, 121), 300.0, 55.0, R.Dilation(3, 2, 1, tile=tile))]
    cams = [scenes.look_at(scenes.orbit_eye(2.6, az, el), width=w, height=h) for (w, h), az, el, _ in spec]
    dils = [d for *_, d in spec]
    targets = [scenes.target_image(c.width, c.height, 7, seed_offset=i + 1) for i, c in enumerate(cams)]
    return U.params_np(s), cams, dils, targets


class Views:
    """Device buffers of every view plus the one-view reference runs."""

    def __init__(self, p32, cams, dils, targets, sh_dtype=torch.float32):
        self.p = U.gpu_params(p32, sh_dtype)
        self.cams, self.dils = cams, dils
        n = self.p.n
        self.grids = [R.gs_grid(c, d) for c, d in zip(cams, dils)]
        self.bufs = []
        for (w_ds, h_ds, tx, ty), t in zip(self.grids, targets):
            self.bufs.append(dict(
                splats=torch.zeros(n, R.SPLAT_FLOATS, device=DEV),
                radii=torch.zeros(n, dtype=torch.int32, device=DEV),
                rects=torch.zeros(n, 4, dtype=torch.int32, device=DEV),
                tiles_touched=torch.zeros(n, dtype=torch.int32, device=DEV),
                ranges=torch.zeros(tx * ty, 2, dtype=torch.int32, device=DEV),
                img=torch.full((h_ds, w_ds, 3), 5.0, device=DEV),
                t_final=torch.full((h_ds, w_ds), 5.0, device=DEV),
                last=torch.full((h_ds, w_ds), 7, dtype=torch.int32, device=DEV),
                target=torch.tensor(t, device=DEV),
                dl_dimg=torch.full((h_ds, w_ds, 3), 5.0, device=DEV),
                grad2d=torch.full((n, R.GRAD2D_FLOATS), 5.0, device=DEV),
                loss=torch.full((1,), 5.0, device=DEV)))

    def table(self):
        fields = set(R.View.__dataclass_fields__) - {"cam", "dil"}
        return R.ViewTable([R.View(c, d, **{k: v for k, v in b.items() if k in fields})
                            for c, d, b in zip(self.cams, self.dils, self.bufs)])

    def project(self):
        p = self.p
        R.gs_project_batch(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, self.table())

    def bin(self):
        n = self.p.n
        for b, (_, _, tx, ty) in zip(self.bufs, self.grids):
            k = int(b["tiles_touched"].to(torch.int64).sum().item())
            ws = torch.empty(R.gs_bin_sort_workspace_size(n, k + 16, tx, ty), dtype=torch.uint8, device=DEV)
            b["sorted_ids"] = torch.empty(k + 16, dtype=torch.int32, device=DEV)
            b["num_pairs"] = torch.zeros(1, dtype=torch.int64, device=DEV)
            R.gs_bin_sort(n, b["rects"], b["tiles_touched"], b["splats"], tx, ty, ws, k + 16, b["sorted_ids"],
                          b["ranges"], b["num_pairs"])
            b["k"] = k
        torch.cuda.synchronize()

    def order(self):
        total = sum(g[2] * g[3] for g in self.grids)
        order = torch.full((total,), -1, dtype=torch.int32, device=DEV)
        R.gs_tile_order_batch(self.table(), order)
        return order


def single_forward(V, i, ppt=0):
    """One-view gs_render_fwd of view i on the batch's lists."""
    b, c, d = V.bufs[i], V.cams[i], V.dils[i]
    w_ds, h_ds, _, _ = V.grids[i]
    img = torch.zeros(h_ds, w_ds, 3, device=DEV)
    tf = torch.zeros(h_ds, w_ds, device=DEV)
    last = torch.zeros(h_ds, w_ds, dtype=torch.int32, device=DEV)
    counts = torch.zeros(3, dtype=torch.int64, device=DEV)
    R.gs_render_fwd(V.p.n, b["splats"], b["sorted_ids"], b["ranges"], c, d, BG, img, tf, last, counts,
                    pixels_per_thread=ppt)
    return img, tf, last, counts


@pytest.fixture(scope="module")
def batch():
    return batch_scene()


def test_project_batch_equals_single_views(batch):
    p32, cams, dils, targets = batch
    V = Views(p32, cams, dils, targets)
    V.project()
    torch.cuda.synchronize()
    p = V.p
    for i, (c, d) in enumerate(zip(cams, dils)):
        n = p.n
        ref = dict(splats=torch.zeros(n, R.SPLAT_FLOATS, device=DEV), radii=torch.zeros(n, dtype=torch.int32, device=DEV),
                   rects=torch.zeros(n, 4, dtype=torch.int32, device=DEV),
                   tiles_touched=torch.zeros(n, dtype=torch.int32, device=DEV))
        R.gs_project(p.means, p.log_scales, p.quats, p.opacity_logits, p.sh_store, c, d, ref["splats"], ref["radii"],
                     ref["rects"], ref["tiles_touched"])
        torch.cuda.synchronize()
        for k, t in ref.items():
            np.testing.assert_array_equal(V.bufs[i][k].cpu().numpy(), t.cpu().numpy(), err_msg=f"view {i} {k}")
        assert int(V.bufs[i]["tiles_touched"].gt(0).sum()) > 100


def test_tile_order_batch_is_a_longest_first_permutation(batch):
    V = Views(*batch)
    V.project()
    V.bin()
    order = V.order().cpu().numpy().astype(np.int64)
    lens = np.concatenate([(b["ranges"][:, 1] - b["ranges"][:, 0]).cpu().numpy() for b in V.bufs])
    assert np.array_equal(np.sort(order), np.arange(lens.size))
    # descending in buckets of 8 per octave of (length + 1): a later entry's
    # length + 1 is at most 9/8 of any earlier entry's
    x = lens[order].astype(np.float64) + 1.0
    assert np.all(x <= np.minimum.accumulate(x) * 1.125 + 1e-9)


@pytest.mark.parametrize("use_order", [False, True])
def test_render_fwd_batch_equals_single_views(batch, use_order):
    V = Views(*batch)
    V.project()
    V.bin()
    order = V.order() if use_order else None
    counts = torch.zeros(3, dtype=torch.int64, device=DEV)
    R.gs_render_fwd_batch(V.p.n, V.table(), BG, tile_order=order, counts=counts)
    torch.cuda.synchronize()
    total = np.zeros(3, np.int64)
    for i in range(len(V.bufs)):
        img, tf, last, c = single_forward(V, i)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(V.bufs[i]["img"].cpu().numpy(), img.cpu().numpy())
        np.testing.assert_array_equal(V.bufs[i]["t_final"].cpu().numpy(), tf.cpu().numpy())
        np.testing.assert_array_equal(V.bufs[i]["last"].cpu().numpy(), last.cpu().numpy())
        total += c.cpu().numpy()
    np.testing.assert_array_equal(counts.cpu().numpy(), total)


def test_batch_view_matches_oracle(batch):
    """View 1 of the batch (257x193, d=2, offset (1,0)) against the FP64 oracle
    on the same lists: image within 1e-4, last index exact, away from the
    oracle's flagged gate decisions."""
    V = Views(*batch)
    V.project()
    V.bin()
    R.gs_render_fwd_batch(V.p.n, V.table(), BG, tile_order=V.order())
    torch.cuda.synchronize()
    i = 1
    p32 = batch[0]
    b, cam, dil = V.bufs[i], V.cams[i], V.dils[i]
    o = orc.project(U.params_f64(p32), orc.as_camera(cam), orc.as_dilation(dil))
    ids = b["sorted_ids"][:b["k"]].cpu().numpy().view(np.uint32)
    ranges = b["ranges"].cpu().numpy().view(np.uint32)
    of = orc.render_fwd(o, ids, ranges, orc.as_camera(cam), orc.as_dilation(dil), BG)
    w_ds, h_ds, tx, ty = V.grids[i]
    tiles_gpu = b["tiles_touched"].cpu().numpy()
    cull_diff = (o["tiles_touched"] > 0) != (tiles_gpu > 0)
    bad = np.zeros(tx * ty, bool)
    rects = b["rects"].cpu().numpy()
    for g in np.nonzero(cull_diff)[0]:
        rc = rects[g] if tiles_gpu[g] > 0 else o["rect"][g]
        for yy in range(rc[1], rc[3] + 1):
            bad[yy * tx + rc[0]: yy * tx + rc[2] + 1] = True
    excl = of["ambiguous"] | U.tile_pixel_mask(bad, w_ds, h_ds, tx, dil.tile)
    # a Gaussian whose culling FP32 and FP64 decide differently (flagged by the
    # oracle: a rect edge or radius within rounding of its threshold) takes
    # its whole rect out of the exact comparison; a few close shell Gaussians
    # cover several of this small view's 56 tiles
    assert excl.mean() < 0.1
    keep = ~excl
    img = b["img"].cpu().numpy().astype(np.float64)
    assert np.abs(img - of["img"])[keep].max() < 1e-4
    np.testing.assert_array_equal(b["last"].cpu().numpy().view(np.uint32)[keep], of["last"][keep])


def test_loss_batch_equals_single_views(batch):
    V = Views(*batch)
    rng = np.random.default_rng(3)
    for b in V.bufs:
        b["img"].copy_(torch.tensor(rng.uniform(0, 1, tuple(b["img"].shape)), dtype=torch.float32))
    R.gs_loss_l1_batch(V.table())
    torch.cuda.synchronize()
    for i, b in enumerate(V.bufs):
        dl = torch.empty_like(b["img"])
        loss = torch.zeros(1, device=DEV)
        R.gs_loss_l1(V.cams[i], V.dils[i], b["img"], b["target"], dl, loss)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(b["dl_dimg"].cpu().numpy(), dl.cpu().numpy())
        L, _ = orc.loss_l1(b["img"].cpu().numpy(), b["target"].cpu().numpy(), orc.as_camera(V.cams[i]),
                           orc.as_dilation(V.dils[i]))
        assert abs(b["loss"].item() - L) < 1e-6 * max(1.0, L)
        assert abs(b["loss"].item() - loss.item()) < 1e-6 * max(1.0, L)


def test_render_fwd_batch_fused_loss_and_zeroing(batch):
    """flags GS_FWD_L1 | GS_FWD_ZERO_GRAD2D: every view's image, dL/dimg and loss as the
    separate batched calls give them, and every view's 2D-gradient rows zeroed."""
    V = Views(*batch)
    V.project()
    V.bin()
    order = V.order()
    R.gs_render_fwd_batch(V.p.n, V.table(), BG, tile_order=order)
    R.gs_loss_l1_batch(V.table())
    torch.cuda.synchronize()
    ref = [(b["img"].clone(), b["dl_dimg"].clone(), b["loss"].item()) for b in V.bufs]
    for b in V.bufs:
        b["img"].fill_(5.0)
        b["dl_dimg"].fill_(5.0)
        b["loss"].fill_(5.0)
        b["grad2d"].fill_(5.0)
    R.gs_render_fwd_batch(V.p.n, V.table(), BG, tile_order=order, flags=R.FWD_L1 | R.FWD_ZERO_GRAD2D)
    torch.cuda.synchronize()
    for b, (img, dl, loss) in zip(V.bufs, ref):
        assert torch.equal(b["img"], img)
        assert torch.equal(b["dl_dimg"], dl)
        assert abs(b["loss"].item() - loss) <= 1e-6 * max(loss, 1e-12)
        assert int(torch.count_nonzero(b["grad2d"]).item()) == 0


def test_render_bwd_batch_equals_single_views(batch):
    V = Views(*batch)
    V.project()
    V.bin()
    t = V.table()
    order = V.order()
    R.gs_render_fwd_batch(V.p.n, t, BG, tile_order=order)
    R.gs_loss_l1_batch(t)
    R.gs_render_bwd_batch(V.p.n, t, BG, tile_order=order, zero_grad2d=True)
    torch.cuda.synchronize()
    for i, b in enumerate(V.bufs):
        g = torch.full_like(b["grad2d"], 9.0)
        R.gs_render_bwd(V.p.n, b["splats"], b["sorted_ids"], b["ranges"], V.cams[i], V.dils[i], BG, b["t_final"],
                        b["last"], b["dl_dimg"], g, zero_grad2d=True)
        torch.cuda.synchronize()
        a, r = b["grad2d"].cpu().numpy(), g.cpu().numpy()
        # float atomics in another order: equal up to FP32 rounding of the sums
        for sl in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
            assert U.max_rel(a[:, sl], r[:, sl]) < 1e-5, (i, sl)
        assert np.all(a[:, 9:] == 0.0)
        assert np.abs(r).max() > 0


def _adam_sets(p, k):
    sets = []
    for _ in range(k):
        ps = [t.clone() for t in p.tensors()]
        sets.append(dict(p=ps, m=[torch.zeros_like(t, dtype=torch.float32) for t in ps],
                         v=[torch.zeros_like(t, dtype=torch.float32) for t in ps],
                         stats=[torch.zeros(p.n, device=DEV), torch.zeros(p.n, device=DEV),
                                torch.zeros(p.n, dtype=torch.int32, device=DEV)]))
    return sets


@pytest.mark.parametrize("sparse,sh_dtype", [(False, torch.float32), (True, torch.float32), (False, torch.bfloat16)],
                         ids=["fp32", "fp32-sparse", "bf16"])
def test_fused_batch_equals_summed_single_views(batch, sparse, sh_dtype):
    """gs_project_bwd_adam_batch = the sum over views of gs_project_bwd, then
    one gs_adam; the densification statistics accumulate once per view. With
    the SH kept only in BF16 both paths round the SH update stochastically with
    the same bits: equal, or one BF16 step apart where their FP32 updates
    straddle a decision."""
    V = Views(*batch, sh_dtype=sh_dtype)
    V.project()
    V.bin()
    t = V.table()
    R.gs_render_fwd_batch(V.p.n, t, BG, tile_order=V.order())
    R.gs_loss_l1_batch(t)
    R.gs_render_bwd_batch(V.p.n, t, BG, zero_grad2d=True)
    torch.cuda.synchronize()
    lrs = [1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3]
    ref, fused = _adam_sets(V.p, 2)
    vis_any = torch.stack([b["tiles_touched"] > 0 for b in V.bufs]).any(0)
    mask = vis_any.to(torch.uint8) if sparse else None
    for step in (1, 2):
        # each step starts both paths from the same state: two trajectories would drift apart by
        # rounding and could then take a colour channel's clamp at zero differently
        for key in ("p", "m", "v"):
            for x, y in zip(ref[key], fused[key]):
                x.copy_(y)
        gsum = gabs = None
        for i, b in enumerate(V.bufs):
            g = [torch.empty_like(x, dtype=torch.float32) for x in ref["p"]]
            R.gs_project_bwd(*ref["p"][:4], ref["p"][4], V.cams[i], V.dils[i], b["tiles_touched"], b["grad2d"], *g,
                             *ref["stats"])
            gsum = g if gsum is None else [x + y for x, y in zip(gsum, g)]
            gabs = [x.abs() for x in g] if gabs is None else [x + y.abs() for x, y in zip(gabs, g)]
        ent = [dict(param=ref["p"][j], grad=gsum[j], m=ref["m"][j], v=ref["v"][j], lr=lrs[j], sr_seed=5)
               for j in range(5)]
        R.gs_adam(ent, 0.9, 0.999, 1e-15, step, row_mask=mask)
        gout = [torch.full_like(x, 7.0, dtype=torch.float32) for x in fused["p"]]
        R.gs_project_bwd_adam_batch(fused["p"], fused["m"], fused["v"], lrs, 0.9, 0.999, 1e-15, step, fused["p"][4],
                                    t, sparse=sparse, pos_acc=fused["stats"][0], col_acc=fused["stats"][1],
                                    count=fused["stats"][2], grads_out=gout, sr_seed=5)
        torch.cuda.synchronize()
        # the views' terms may cancel: the rounding of their sum is bounded relative to the sum
        # of their magnitudes, and the two paths round it in different orders
        for x, y, z in zip(gout, gsum, gabs):
            err = np.abs(x.cpu().numpy().astype(np.float64) - y.cpu().numpy()).max()
            assert err <= 1e-5 * float(z.max().item()), err
    for key, rtol in (("p", 1e-6), ("m", 1e-5), ("v", 1e-5), ("stats", 1e-6)):
        for i, (x, y) in enumerate(zip(ref[key], fused[key])):
            a, b = x.float().cpu().numpy(), y.float().cpu().numpy()
            if key == "p" and i == 4 and sh_dtype != torch.float32:
                assert (a == b).mean() >= 0.999
                step_ = np.abs(b) * 2.0 ** -7 + 1e-38  # a BF16 step at |b| is at most this
                assert (np.abs(a - b) <= step_).all()
                assert (b != V.p.sh_store.float().cpu().numpy()).mean() > 0.05
                continue
            assert U.max_rel(a, b) < rtol, key
    cnt = fused["stats"][2].cpu().numpy()
    assert cnt.max() >= 2  # some Gaussians are seen in several views
    if sparse:
        hidden = ~vis_any.cpu().numpy()
        assert hidden.any()
        before = V.p.means.cpu().numpy()
        np.testing.assert_array_equal(fused["p"][0].cpu().numpy()[hidden], before[hidden])
        assert np.all(fused["m"][0].cpu().numpy()[hidden] == 0.0)


def test_device_step_counter_matches_host_step(batch):
    """gs_adam_advance + bias_dev (what a captured graph replays) gives the
    steps the host-side step count gives."""
    p32, cams, dils, targets = batch
    V = Views(p32, cams[:1], dils[:1], targets[:1])
    V.project()
    V.bin()
    t = V.table()
    R.gs_render_fwd_batch(V.p.n, t, BG)
    R.gs_loss_l1_batch(t)
    R.gs_render_bwd_batch(V.p.n, t, BG, zero_grad2d=True)
    lrs = [1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3]
    host, dev = _adam_sets(V.p, 2)
    step_dev = torch.zeros(1, dtype=torch.int32, device=DEV)
    bias = torch.zeros(2, device=DEV)
    b = V.bufs[0]
    for step in (1, 2, 3):
        R.gs_project_bwd_adam(host["p"], host["m"], host["v"], lrs, 0.9, 0.999, 1e-15, step, host["p"][4], cams[0],
                              dils[0], b["tiles_touched"], b["grad2d"])
        R.gs_adam_advance(step_dev, 0.9, 0.999, bias)
        R.gs_project_bwd_adam(dev["p"], dev["m"], dev["v"], lrs, 0.9, 0.999, 1e-15, 0, dev["p"][4], cams[0],
                              dils[0], b["tiles_touched"], b["grad2d"], bias_dev=bias)
        torch.cuda.synchronize()
        assert step_dev.item() == step
        # the betas are FP32 arguments: the corrections use their FP32 values
        b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))
        want = np.array([1 / (1 - b1 ** step), 1 / (1 - b2 ** step)], np.float32)
        got = bias.cpu().numpy()
        assert np.all(np.abs(got - want) <= np.spacing(want))
    for key in ("p", "m", "v"):
        for x, y in zip(host[key], dev[key]):
            assert U.max_rel(x.cpu().numpy(), y.cpu().numpy()) < 1e-6, key


def _state(st):
    return [st.step_dev, st.bias_dev, st.pos_acc, st.col_acc, st.vis_count] + st.p.tensors() + st.m + st.v


def test_batch_train_step_graph_replay_equals_eager(batch):
    """A replayed CUDA graph of BatchTrainStep (d=2, rotating offsets) takes
    the step the eager calls take from the same state: forward outputs bit for
    bit, the device step counter, and the parameters up to what float atomics
    in another order can change (Adam turns the sign of a near-zero gradient
    into a full +-lr step, so a few elements may differ by up to 2 lr)."""
    p32, cams, _, targets = batch
    tg = [torch.tensor(t, device=DEV) for t in targets]
    p = U.gpu_params(p32)
    st = BatchTrainStep(p, cams, tg, d=2, adam=AdamConfig(lr_means=1e-3))
    st.capture()  # one eager step per phase, then one graph per phase
    torch.cuda.synchronize()
    assert st.step_dev.item() == st.phases
    # odd image sizes change a view's tile grid with the offset: the list-length order every step
    assert not st.reuse_order and not st._bwd_order_ok
    lrs = [st.adam.lr_means, st.adam.lr_log_scales, st.adam.lr_quats, st.adam.lr_opacity, st.adam.lr_sh]
    for ph in range(st.phases):
        snap = [t.clone() for t in _state(st)]
        st.run(ph)
        torch.cuda.synchronize()
        eager = dict(img=[x.clone() for x in st.img], last=[x.clone() for x in st.last],
                     tf=[x.clone() for x in st.t_final], loss=st.loss.clone(), step=st.step_dev.item(),
                     params=[t.clone() for t in p.tensors()])
        for t, s0 in zip(_state(st), snap):
            t.copy_(s0)
        st.graphs[ph].replay()
        torch.cuda.synchronize()
        assert st.step_dev.item() == eager["step"] == snap[0].item() + 1
        for i in range(st.V):
            assert torch.equal(st.img[i], eager["img"][i]), (ph, i)
            assert torch.equal(st.last[i], eager["last"][i]), (ph, i)
            assert torch.equal(st.t_final[i], eager["tf"][i]), (ph, i)
        np.testing.assert_allclose(st.loss.cpu().numpy(), eager["loss"].cpu().numpy(), rtol=1e-5)
        for t, e, p0, lr in zip(p.tensors(), eager["params"], snap[5:10], lrs):
            diff = (t - e).abs()
            assert diff.max().item() <= 2.0 * lr * 1.01 + 1e-6
            assert (diff > 1e-6 * (1.0 + e.abs())).float().mean().item() < 0.01
            assert (t != p0).any()  # the step moved the parameters
    # the offsets rotate: view 0 renders a different lattice in each phase
    imgs = []
    for _ in range(st.phases):
        st.step()
        torch.cuda.synchronize()
        imgs.append(st.img[0].clone())
    assert not torch.equal(imgs[0], imgs[1])
    assert st.step_dev.item() == 3 * st.phases
    assert not st.overflowed()


def test_batch_forward_in_the_previous_backward_order():
    """Views whose tile grids do not change with the offset: after the first phase the
    batched forward launches in the previous backward's order (no order kernel), with
    results bit-identical to the list-length order."""
    s = scenes.cluster_scene(20000, index=8, log_scale_mean=-3.6)
    cams = [scenes.look_at(scenes.orbit_eye(2.6, az, 20.0), width=w, height=h)
            for (w, h), az in (((256, 128), 20.0), ((192, 160), 140.0), ((320, 192), 260.0))]
    tg = [torch.tensor(scenes.quantize_u8(scenes.target_image(c.width, c.height, 8, seed_offset=i + 1)), device=DEV)
          for i, c in enumerate(cams)]
    p32 = U.params_np(s)
    p = U.gpu_params(p32)
    st = BatchTrainStep(p, cams, tg, d=2)
    assert st.reuse_order
    st.run(0)
    assert st._bwd_order_ok
    snap = [t.clone() for t in p.tensors()]
    st.run(1)  # its forward launches in the order the phase-0 backward made
    torch.cuda.synchronize()
    imgs = [x.clone() for x in st.img]
    lasts = [x.clone() for x in st.last]
    ref = BatchTrainStep(GaussianParams(*snap, snap[4]), cams, tg, d=2)
    assert not ref._bwd_order_ok
    ref.render_pass(1)  # the list-length order
    torch.cuda.synchronize()
    for i in range(len(cams)):
        assert torch.equal(imgs[i], ref.img[i]), i
        assert torch.equal(lasts[i], ref.last[i]), i


def test_batch_train_step_reduces_loss(batch):
    p32, cams, _, targets = batch
    # fit the batch to renders of a perturbed copy of the scene
    tg = [torch.tensor(t, device=DEV) for t in targets]
    p = U.gpu_params(p32)
    st = BatchTrainStep(p, cams, tg, d=1, adam=AdamConfig(lr_sh=1e-2, lr_opacity=5e-2))
    st.run(0)
    l0 = st.loss.sum().item()
    for _ in range(20):
        st.step()
    torch.cuda.synchronize()
    assert st.loss.sum().item() < l0


def test_autotune_returns_a_measured_candidate(batch):
    p32, cams, _, targets = batch
    tg = [torch.tensor(t, device=DEV) for t in targets]
    p = U.gpu_params(p32)
    before = [t.clone() for t in p.tensors()]
    best, times = autotune_batch(p, cams[:2], tg[:2], d=2, candidates=((8, 1), (16, 2), (32, 4)), iters=1)
    assert best in times and len(times) == 3 and all(v > 0 for v in times.values())
    for x, y in zip(before, p.tensors()):
        assert torch.equal(x, y)  # tuning does not touch the parameters
