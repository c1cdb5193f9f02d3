"""Whole-network pins of the oracle (CPU only).

* The layer table it reads the blob with matches Table 3 (tests/golden/table3_layers.txt):
  operation, stride, output channels, activation, and the resolution ratio that
  results from walking the shapes; the input channel counts chain consistently.
* An independent float64 composition of the forward from torch.nn.functional
  library routines (conv2d, conv_transpose2d, avg_pool2d, interpolate,
  grid_sample, sigmoid) agrees to 1e-9 at two sizes (one needing the pad to 16).
* Circular mode: shifting both inputs cyclically by multiples of 16 pixels
  shifts the output by the same amount, bit for bit.
* Sanity of the intermediates: mask logits and flows finite, output in [0, 1].
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

import oracle
from synth import scene, weights

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_layers.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        sub, op, stride, ratio, co, act = line.split()
        rows.append((sub, op, int(stride), ratio, int(co), act))
    return rows


def _ratio(text, i):
    if text.startswith("2^i/"):
        return Fraction(2 ** i, int(text[4:]))
    return Fraction(text)


def test_layer_table_matches_table3():
    table = oracle.layer_table()
    gold = _golden_rows()
    vib, ctx, ref = gold[:10], gold[10:18], gold[18:]
    expect = []
    for i in range(3):
        expect += [(f"vib{i}", r, _ratio(r[3], i)) for r in vib]
    expect += [("ctx", r, _ratio(r[3], 0)) for r in ctx]
    expect += [("ref", r, _ratio(r[3], 0)) for r in ref]
    assert len(table) == len(expect) == 51
    # walk the resolutions: VIB_i input at 2^i/4, ContextNet on the full frame,
    # RefineNet encoder on the full frame (its decoders go back up)
    res = {}
    for (name, kind, ci, co, stride, relu), (sub, g, ratio) in zip(table, expect):
        assert name.startswith(sub)
        assert kind == g[1] and stride == g[2] and co == g[4], name
        assert relu == (g[5] == "relu"), name
        prev = res.get(sub, Fraction(2 ** int(sub[3]), 4) if sub.startswith("vib") else Fraction(1))
        now = prev * 2 if kind == "convT" else prev / stride
        assert now == ratio, (name, now, ratio)
        res[sub] = now
    # the blob generator and the oracle agree on the manifest
    assert [(n, k, ci, co, s, r) for n, k, ci, co, s, r in table] == weights.manifest()
    assert oracle.n_floats() == weights.n_floats() == 16407874


def test_input_channels_chain():
    t = {n: (ci, co) for n, _, ci, co, _, _ in oracle.layer_table()}
    for i in range(3):
        names = [f"vib{i}.c0", f"vib{i}.c1"] + [f"vib{i}.m{k}" for k in range(6)] + [f"vib{i}.t0", f"vib{i}.t1"]
        for a, b in zip(names, names[1:]):
            assert t[a][1] == t[b][0]
    ctxc = [t[f"ctx.c{k}"][1] for k in (1, 3, 5, 7)]
    enc = [t[f"ref.e{k}b"][1] for k in range(4)]
    # encoder k+1 takes [e_k, left ctx_k, right ctx_k]; d0 takes [e3, ctx_3 x 2]
    for k in range(3):
        assert t[f"ref.e{k + 1}a"][0] == enc[k] + 2 * ctxc[k]
    assert t["ref.d0"][0] == enc[3] + 2 * ctxc[3]
    dec = [t[f"ref.d{k}"][1] for k in range(4)]
    for k in range(1, 4):
        assert t[f"ref.d{k}"][0] == dec[k - 1] + enc[3 - k]
    assert t["ref.out"][0] == dec[3]


# ---------------------------------------------------------------------------
# independent torch.nn.functional composition (zero mode)

def _torch_forward(blob, left, right, t):
    L = {k: (torch.from_numpy(np.array(w, np.float64)), torch.from_numpy(np.array(b, np.float64)))
         for k, (w, b) in weights.layer_views(blob).items()}
    kinds = {n: (k, s, r) for n, k, _, _, s, r in weights.manifest()}

    def layer(name, x):
        kind, s, relu = kinds[name]
        w, b = L[name]
        y = Fn.conv2d(x, w, b, stride=s, padding=1) if kind == "conv" else \
            Fn.conv_transpose2d(x, w, b, stride=2, padding=1)
        return torch.relu(y) if relu else y

    def vib(i, x):
        for n in ["c0", "c1"] + [f"m{k}" for k in range(6)] + ["t0", "t1"]:
            x = layer(f"vib{i}.{n}", x)
        return x

    def warp(img, flow):
        _, _, H, W = img.shape
        ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64),
                                torch.arange(W, dtype=torch.float64), indexing="ij")
        gx = (xs + flow[:, 0] + 0.5) / W * 2 - 1
        gy = (ys + flow[:, 1] + 0.5) / H * 2 - 1
        return Fn.grid_sample(img, torch.stack([gx, gy], -1), mode="bilinear",
                              padding_mode="border", align_corners=False)

    H, W, _ = left.shape
    Hp, Wp = -(-H // 16) * 16, -(-W // 16) * 16
    Il, Ir = [Fn.pad(torch.from_numpy(np.array(a, np.float64)).permute(2, 0, 1)[None],
                     (0, Wp - W, 0, Hp - H)) for a in (left, right)]
    pyr = {2: (Il, Ir), 1: (Fn.avg_pool2d(Il, 2), Fn.avg_pool2d(Ir, 2)),
           0: (Fn.avg_pool2d(Il, 4), Fn.avg_pool2d(Ir, 4))}
    a, b = pyr[0]
    out = vib(0, torch.cat([a, b, torch.full_like(a[:, :1], t)], 1))
    for s in (1, 2):
        up = Fn.interpolate(out, scale_factor=2, mode="bilinear", align_corners=False)
        F, M = up[:, :4] * 2, up[:, 4:5]
        a, b = pyr[s]
        x = torch.cat([a, b, warp(a, F[:, :2]), warp(b, F[:, 2:4]), M, F, torch.full_like(M, t)], 1)
        out = torch.cat([F, M], 1) + vib(s, x)
    Ilm, Irm = warp(Il, out[:, :2]), warp(Ir, out[:, 2:4])
    M = torch.sigmoid(out[:, 4:5])
    Ib = M * Ilm + (1 - M) * Irm
    ctx = []
    for img in (Il, Ir):
        x, lv = img, []
        for k in range(8):
            x = layer(f"ctx.c{k}", x)
            if k % 2:
                lv.append(x)
        ctx.append(lv)
    Fk, cw = out[:, :4], []
    for k in range(4):
        Fk = Fn.avg_pool2d(Fk, 2) * 0.5
        cw.append((warp(ctx[0][k], Fk[:, :2]), warp(ctx[1][k], Fk[:, 2:4])))
    x, enc = torch.cat([Ilm, Irm], 1), []
    for k in range(4):
        x = layer(f"ref.e{k}b", layer(f"ref.e{k}a", x))
        enc.append(x)
        x = torch.cat([x, cw[k][0], cw[k][1]], 1)
    d = layer("ref.d0", x)
    for k in range(1, 4):
        d = layer(f"ref.d{k}", torch.cat([d, enc[3 - k]], 1))
    z = layer("ref.out", d)
    y = torch.clamp(Ib + 2 * torch.sigmoid(z) - 1, 0, 1)
    return y[0, :, :H, :W].permute(1, 2, 0).numpy(), out[0].permute(1, 2, 0).numpy()


@pytest.mark.parametrize("H,W,t,seed", [(64, 64, 0.5, 1), (40, 56, 0.3, 2)])
def test_forward_matches_torch_composition(H, W, t, seed):
    blob = weights.he_init(0)
    left, right = scene.stereo_pair(seed, H, W, max_disp=6.0)
    got, d = oracle.vinet_forward(blob, left, right, t, dumps=True)
    ref, ref_flow = _torch_forward(blob, left, right, t)
    np.testing.assert_allclose(d["vib2"], ref_flow, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)
    assert np.isfinite(d["vib2"]).all() and got.min() >= 0 and got.max() <= 1
    # the output is not trivially clamped everywhere
    assert ((got > 0) & (got < 1)).mean() > 0.5


def test_forward_circular_shift_equivariance():
    blob = weights.he_init(0)
    left, right = scene.stereo_pair(3, 64, 48, max_disp=6.0)
    a = oracle.vinet_forward(blob, left, right, 0.5, circ=True)
    sh = (16, -32)
    b = oracle.vinet_forward(blob, np.roll(left, sh, (0, 1)), np.roll(right, sh, (0, 1)), 0.5, circ=True)
    np.testing.assert_array_equal(np.roll(a, sh, (0, 1)), b)


def test_forward_t_changes_output_and_rejects_bad_sizes():
    blob = weights.he_init(0)
    left, right = scene.stereo_pair(4, 32, 32, max_disp=4.0)
    a = oracle.vinet_forward(blob, left, right, 0.25)
    b = oracle.vinet_forward(blob, left, right, 0.75)
    assert np.abs(a - b).max() > 1e-6
    with pytest.raises(ValueError):
        oracle.vinet_forward(blob[:-1], left, right, 0.5)
    with pytest.raises(ValueError):  # circular mode needs multiples of 16
        oracle.vinet_forward(blob, left[:30], right[:30], 0.5, circ=True)
