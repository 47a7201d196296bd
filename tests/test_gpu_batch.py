"""Batched serving through the C ABI (rw_batch_*): images of uneven sizes and label counts,
solved in one call over several streams, then rounds of added seeds captured into a CUDA graph
and replayed (the graph updated in place between rounds).  Every item must equal the same
solve run alone, bit for bit, and the FP64 oracle pipeline on the same basis within 1e-3; the
launch-shape table changes only the order of the projection's partial sums."""
import numpy as np
import pytest

import synth
from oracle import eig, graph, pipeline
from tests.gpu_common import TOL_PROB, dev, f32, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")

SHAPES = [((48, 48), 2), ((40, 56), 3), ((64, 36), 4), ((56, 44), 5), ((32, 60), 2)]
M = 40


@pytest.fixture(scope="module")
def images():
    from paper_1607_04174_gb300 import build
    build.build()
    out = []
    for k, (dims, L) in enumerate(SHAPES):
        J, _, truth = synth.voronoi_image(dims[0], dims[1], n_regions=L, seed=synth.BASE_SEED + 50 + k)
        J = f32(J)
        go = graph.build_graph(J, dims, 90.0)
        lam, Q = eig.smallest_eigpairs(go.Lhat, M)
        g = rw.rw_build_graph(to_dev(J, torch.float32), dims, 90.0)
        b = rw.rw_basis_create(g, to_dev(f32(Q), torch.float32), lam)
        # eight rounds of seeds: round r uses the first 3 (r + 1) seeds per label
        si, sl = synth.sample_seeds(truth, dims, 24, 2, seed=synth.BASE_SEED + 70 + k)
        rounds = []
        for r in range(8):
            take = np.concatenate([np.nonzero(sl == c)[0][:3 * (r + 1)] for c in range(L)])
            rounds.append((si[take].copy(), sl[take].copy()))
        out.append(dict(dims=dims, L=L, go=go, Q=f32(Q), lam=lam, g=g, b=b, rounds=rounds,
                        N=go.N))
    yield out
    for im in out:
        rw.rw_basis_free(im["b"])
        rw.rw_graph_free(im["g"])


def _items(images, r, share_last=False):
    items = []
    for im in images:
        si, sl = im["rounds"][r]
        items.append(dict(g=im["g"], b=im["b"], seed_idx=to_dev(si), seed_lab=to_dev(sl),
                          n_labels=im["L"], prob=torch.empty(im["N"], im["L"], device=dev()),
                          labels=torch.empty(im["N"], dtype=torch.uint8, device=dev())))
    if share_last:   # a second session on the first image (same graph handle)
        im = images[0]
        si, sl = im["rounds"][max(r - 1, 0)]
        items.append(dict(g=im["g"], b=im["b"], seed_idx=to_dev(si), seed_lab=to_dev(sl),
                          n_labels=im["L"], prob=torch.empty(im["N"], im["L"], device=dev()),
                          labels=torch.empty(im["N"], dtype=torch.uint8, device=dev())))
    return items


def _alone(it, m=0):
    prob = torch.empty_like(it["prob"])
    lab = torch.empty_like(it["labels"])
    rw.rw_solve(it["g"], it["b"], it["seed_idx"], it["seed_lab"], it["n_labels"], prob, lab,
                m=m, want_info=False)
    return prob.cpu().numpy(), lab.cpu().numpy()


def test_batch_equals_single_solves_and_oracle(images):
    bt = rw.rw_batch_create(4)
    try:
        items = _items(images, 3, share_last=True)
        rw.rw_batch_solve(bt, items, m=30)   # a fixed m, so the oracle runs the same pipeline
        torch.cuda.synchronize()
        got = [(it["prob"].cpu().numpy(), it["labels"].cpu().numpy()) for it in items]
        for it, (p, l) in zip(items, got):
            pa, la = _alone(it, m=30)
            np.testing.assert_array_equal(p, pa)
            np.testing.assert_array_equal(l, la)
        for im, (p, _) in zip(images, got):
            si, sl = im["rounds"][3]
            ref = pipeline.online_solve(im["go"], im["Q"], im["lam"], si, sl, im["L"],
                                        gamma=1e-3, m=30, refine_steps=3)
            assert np.abs(p - ref["U"]).max() <= TOL_PROB
    finally:
        rw.rw_batch_free(bt)


def test_captured_rounds_replay_and_update_in_place(images):
    bt = rw.rw_batch_create(4)
    stream = torch.cuda.Stream()
    try:
        # size every workspace with the last round's seed count (uncaptured)
        for it in _items(images, 7):
            _alone(it)
        updates = []
        with torch.cuda.stream(stream):
            for r in range(8):
                items = _items(images, r)
                updates.append(rw.rw_batch_capture(bt, items, stream=stream))
                rw.rw_batch_launch(bt, stream=stream)
                stream.synchronize()
                for it in items:
                    pa, la = _alone(it)
                    np.testing.assert_array_equal(it["prob"].cpu().numpy(), pa)
                    np.testing.assert_array_equal(it["labels"].cpu().numpy(), la)
        assert updates[0] == 0
        print("graph updated in place on rounds:", updates)
        assert sum(updates[1:]) >= 1
    finally:
        rw.rw_batch_free(bt)


def test_launch_shapes_keep_parity(images):
    try:
        for proj, back in ((1, 1), (4, 2)):
            rw.rw_set_launch_shape(1 << 30, proj, back)
            for im in images[:2]:
                si, sl = im["rounds"][5]
                prob = torch.empty(im["N"], im["L"], device=dev())
                rw.rw_solve(im["g"], im["b"], to_dev(si), to_dev(sl), im["L"], prob, m=30,
                            want_info=False)
                ref = pipeline.online_solve(im["go"], im["Q"], im["lam"], si, sl, im["L"],
                                            gamma=1e-3, m=30, refine_steps=3)
                assert np.abs(prob.cpu().numpy() - ref["U"]).max() <= TOL_PROB
    finally:
        rw.rw_set_launch_shape(0, 1, 1)


def test_batch_rejects_bad_items(images):
    bt = rw.rw_batch_create(2)
    try:
        items = _items(images, 0)
        items[1]["n_labels"] = 0
        with pytest.raises(rw.RWError) as e:
            rw.rw_batch_solve(bt, items)
        assert e.value.status == rw.RW_ERR_INVALID_ARG
        with pytest.raises(rw.RWError):
            rw.rw_batch_launch(bt)   # nothing captured yet
    finally:
        rw.rw_batch_free(bt)
