"""Learned proposal on the GPU against the fp64 oracle (oracle/cnn.py):
thumbnails, forward, backward, the Adam update in closed form, the proposal's
top-k / tau masks and its use by lfc_compress.

The oracle stores BF16 where the network's stated precision puts BF16
(inputs, convolution weights, activations, pre-activation gradients) and
accumulates in fp64; the GPU accumulates in FP32. Every probability and every
gradient element is compared on its own: within 1e-2 of its value plus 1e-3 of
the largest magnitude in its tensor (the floor covers elements that cancel to
near zero, where FP32 accumulation order and a rare BF16 re-rounding or ReLU
mask flip dominate)."""
import numpy as np
import pytest

import oracle
from oracle import cnn as ocnn
from paper_2310_09467_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2310_09467_gb300 import build, lfc
    build.build()
    return lfc


def test_thumbnails_match_oracle(L):
    frs = [(synth.beads(390, 390, 15, peak=2000.0, seed=3), 15), (synth.cells(1300, 1300, 13, seed=4), 13)]
    net = L.Cnn(26, 2)
    for fr, p in frs:
        th = net.thumbnails([L.to_device_frame(fr)], p, want=True).cpu().numpy()[0]
        ref = ocnn.thumbnail(fr, p)
        assert np.max(np.abs(th - ref)) < 2e-5


def _rand_case(seed, n):
    rng = np.random.default_rng(seed)
    P = ocnn.init_params(32, 26, seed=seed)
    for k in P:
        if k.startswith("b"):
            P[k] = 0.05 * rng.normal(size=P[k].shape)
    x = np.zeros((n, 2, 256, 256))
    x[:, :, :200, :230] = rng.uniform(0, 1.2, size=(n, 2, 200, 230))
    return P, x


def test_forward_and_backward_match_oracle(L):
    import torch
    n = 2
    P, x = _rand_case(5, n)
    net = L.Cnn(26, n)
    net.set_params(net.flat_from_dict(P))
    net.set_thumbnails(torch.from_numpy(x.astype(np.float32)).cuda())
    probs = net.forward(n).cpu().numpy()
    Pr = {k: (ocnn.bf16(v) if k.startswith("w") and k != "wl" else v) for k, v in P.items()}
    xr = ocnn.bf16(x)
    labels = np.array([3, 17], dtype=np.int32)
    ref_p, ref_g = [], None
    for b in range(n):
        logits, _ = ocnn.forward(Pr, xr[b], ocnn.bf16)
        ref_p.append(ocnn.softmax(logits))
        g = ocnn.backward(Pr, xr[b], int(labels[b]), ocnn.bf16)
        ref_g = g if ref_g is None else {k: ref_g[k] + g[k] for k in g}
    ref_p = np.array(ref_p)
    bad = np.abs(probs - ref_p) > 1e-2 * ref_p + 1e-5
    assert not bad.any(), ("probs", int(bad.sum()), float(np.max(np.abs(probs - ref_p) / (ref_p + 1e-5))))
    loss = net.backward(torch.from_numpy(labels).cuda()).cpu().numpy()
    ref_loss = np.array([-np.log(ref_p[b][labels[b]]) for b in range(n)])
    assert np.all(np.abs(loss - ref_loss) <= 1e-2 * ref_loss + 1e-5), (loss, ref_loss)
    _, g = net.get_params(grads=True)
    G = net.dict_from_flat(g)
    for k in ref_g:
        r = ref_g[k] / n
        bound = 1e-2 * np.abs(r) + 1e-3 * np.abs(r).max()
        err = np.abs(G[k] - r)
        worst = int(np.argmax(err / bound))
        assert np.all(err <= bound), (k, int((err > bound).sum()), r.size, float(err.flat[worst]),
                                      float(r.flat[worst]), float(np.abs(r).max()))


def test_adam_step_closed_form(L):
    import torch
    n = 1
    P, x = _rand_case(7, n)
    net = L.Cnn(26, n)
    flat = net.flat_from_dict(P)
    net.set_params(flat)
    net.set_thumbnails(torch.from_numpy(x.astype(np.float32)).cuda())
    net.backward(torch.tensor([4], dtype=torch.int32, device="cuda"))
    p0, g = net.get_params(grads=True)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    net.adam_step(lr, b1, b2, eps)
    p1 = net.get_params()
    m = (1 - b1) * g.astype(np.float64)
    v = (1 - b2) * g.astype(np.float64) ** 2
    exp = p0 - lr * (m / (1 - b1)) / (np.sqrt(v / (1 - b2)) + eps)
    assert np.allclose(p1, exp, rtol=1e-4, atol=1e-6)


def test_training_reduces_loss(L):
    import torch
    n = 4
    _, x = _rand_case(9, n)
    net = L.Cnn(26, n, seed=11)
    net.set_thumbnails(torch.from_numpy(x.astype(np.float32)).cuda())
    labels = torch.tensor([1, 5, 9, 20], dtype=torch.int32, device="cuda")
    first = float(net.backward(labels).mean())
    for _ in range(40):
        net.backward(labels)
        net.adam_step(3e-3)
    last = float(net.backward(labels).mean())
    assert last < 0.5 * first, (first, last)


def test_proposal_masks_and_compress(L):
    import torch
    fr, p = synth.beads(390, 390, 15, peak=2000.0, seed=21), 15
    d = L.to_device_frame(fr)
    plan = L.Plan(390, 390, 15, block_bytes=30000)
    ids = oracle.default_ids()
    net = L.Cnn(len(ids), 4, seed=3)
    net.thumbnails([d], p)
    probs = net.forward(1).cpu().numpy()[0]
    top3 = set(np.argsort(-probs, kind="stable")[:3])
    plan.set_proposal(net, ids, 3, 0.0)
    m = plan.propose([d], p).cpu().numpy().view(np.uint64)[0]
    got = {k for k, cid in enumerate(ids) if (int(m[cid >> 6]) >> (cid & 63)) & 1}
    assert got == top3
    # judged on the proposed ids only: the choice is the best of those
    ch, sc = plan.judge([d], p)
    best_all, scores = oracle.judge(fr, p, ids)
    cand = [ids[k] for k in top3]
    exp = max(cand, key=lambda c: (scores[ids.index(c)], -c))
    assert int(ch.cpu()[0]) == exp
    blob = plan.compress_to_bytes([d], p)[0]
    assert blob == oracle.compress_id(fr, p, exp, block_bytes=30000)
    # tau above 1: always the exhaustive judge
    plan.set_proposal(net, ids, 1, 1.5)
    blob2 = plan.compress_to_bytes([d], p)[0]
    assert blob2 == oracle.compress_id(fr, p, best_all, block_bytes=30000)
