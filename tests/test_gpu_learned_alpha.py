"""Learned alpha: GPU gradients against the CPU FP64 oracle, spectrum features
against a direct computation, and what training gains over the a-priori rule."""
import numpy as np
import pytest

import bhcp_inputs as bi
from oracle.mlp_oracle import adam_update, bf16_round, mlp_loss_and_grads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2107_06381_gb300 as Q  # noqa: E402
from paper_2107_06381_gb300 import learned_alpha as LA  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    Q.build_library()
    Q.load_library()


def _oracle_params(mlp, flat):
    """The oracle evaluates the network with the bf16 weights the kernels use
    (biases stay FP32) and with the standardisation folded into the input."""
    p = mlp.unpack(flat)
    for k in ("W1", "W2", "w3"):
        p[k] = bf16_round(p[k].astype(np.float32))
    return p


def test_gradients_match_oracle():
    rng = np.random.default_rng(0)
    B, K, N = 96, LA.IN_DIM, 128
    mlp = Q.MLP(K, N, max_batch=256, seed=3)
    mean = rng.normal(size=K).astype(np.float32)
    sd = rng.uniform(0.5, 2.0, size=K).astype(np.float32)
    mlp.set_norm(mean, sd)
    x = rng.normal(size=(B, K)).astype(np.float32)
    t = rng.normal(size=B).astype(np.float32)
    xd = torch.as_tensor(x).cuda()
    td = torch.as_tensor(t).cuda()
    loss, g = mlp.gradients(xd, td)
    flat, _, _, _ = mlp.get_params()
    p = _oracle_params(mlp, flat)
    xs = (x.astype(np.float64) - mean) * (1.0 / sd.astype(np.float64))
    want_loss, want = mlp_loss_and_grads(p, xs, t)
    got = mlp.unpack(g)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss)
    for k in want:
        np.testing.assert_allclose(got[k], want[k], rtol=2e-3, atol=2e-4 * np.abs(want[k]).max() + 1e-9, err_msg=k)
    # one Adam step matches the oracle's update of the FP32 master weights
    mlp.train_step(xd, td, 1e-2)
    after, m, v, step = mlp.get_params()
    want_p, _, _ = adam_update(flat.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, 1e-2)
    assert step == 1
    np.testing.assert_allclose(after, want_p, rtol=1e-5, atol=1e-6)
    mlp.close()


def test_features_match_direct_spectrum():
    grid, z0, gd, delta = bi.alpha_training_batch(3, seed=7, M=64, nt=32)
    g = torch.as_tensor(gd.reshape(3, -1), dtype=torch.float64).cuda()
    feats = torch.empty((3, LA.IN_DIM), dtype=torch.float32, device="cuda")
    fp = Q.Features(64, grid.T, grid.nt, 8)
    fp.run(g, delta, feats)
    got = feats.cpu().numpy()
    fp.close()
    n = 63
    j = np.arange(1, n + 1)
    S = np.sin(np.pi * np.outer(j, j) / 64)
    kx, ky = np.meshgrid(j, j)
    bins = np.minimum(63, np.floor(64 * np.sqrt(kx ** 2 + ky ** 2) / (np.sqrt(2) * 64)).astype(int))
    for b in range(3):
        c = (S @ gd[b] @ S) * (2.0 / 64) ** 2            # sine-series coefficients of g_delta
        want = np.full(64, -30.0)
        for k in range(64):
            sel = bins == k
            if sel.any():
                want[k] = np.log10(np.mean(c[sel] ** 2) + 1e-30)
        np.testing.assert_allclose(got[b, :64], want, rtol=0, atol=2e-3)
        np.testing.assert_allclose(got[b, 64:], [np.log10(delta[b]), grid.T, np.log2(grid.nt)], rtol=1e-6)


@pytest.mark.parametrize("scale", [2.0 ** -1000, 2.0 ** -80, 2.0 ** 60, 2.0 ** 600], ids=["1e-301", "1e-24", "1e18", "4e180"])
def test_features_at_any_data_scale(scale):
    """The spectrum is taken of g scaled by the power of two nearest 1/delta, so
    the FP32 DSTs and squares stay in range: the features of s g (with s delta)
    are those of g with the bins moved by log10 s^2, down to the 1e-30 floor of
    their definition."""
    grid, z0, gd, delta = bi.alpha_training_batch(2, seed=8, M=64, nt=32)
    fp = Q.Features(64, grid.T, grid.nt, 8)
    out = []
    for sc in (1.0, scale):
        g = torch.as_tensor(gd.reshape(2, -1) * sc, dtype=torch.float64).cuda()
        feats = torch.empty((2, LA.IN_DIM), dtype=torch.float32, device="cuda")
        fp.run(g, np.asarray(delta) * sc, feats)
        out.append(feats.cpu().numpy().astype(np.float64))
    fp.close()
    base, got = out
    want = np.maximum(base[:, :64] + 2 * np.log10(scale), -30.0)
    occupied = base[:, :64] > -29.0                      # bins holding modes (bin 0 holds none)
    assert np.isfinite(got).all()
    np.testing.assert_allclose(got[:, :64][occupied], want[occupied], rtol=0, atol=1e-3)
    np.testing.assert_allclose(got[:, 64], np.log10(np.asarray(delta) * scale), rtol=1e-6)


def test_training_beats_the_a_priori_rule(tmp_path):
    """Trained on 8192 method-labelled instances (2D 127^2 x 128), the network's
    alpha reconstructs 1024 held-out instances better than alpha = delta."""
    data = LA.make_dataset(8192, seed=1, chunk=4096)
    mlp, hist = LA.train(data, epochs=25, batch=512, lr=2e-3, seed=0)
    assert hist[-1][1] < hist[0][1]
    ev = LA.evaluate(mlp, 1024, seed=2, chunk=1024)
    learned, rule, best = ev["learned"].mean(), ev["rule"].mean(), ev["best"].mean()
    print(f"mean e_h: learned {learned:.4f}  a-priori {rule:.4f}  discrepancy {ev['morozov'].mean():.4f}  "
          f"best-of-scan {best:.4f}; one-alpha solves/s {ev['one_alpha_solves_per_s']:.0f}, "
          f"scan solves/s {ev['scan_solves_per_s']:.0f}")
    assert learned < rule
    assert learned >= best * (1 - 1e-6)
    # checkpoint round trip
    path = str(tmp_path / "mlp.npz")
    LA.save_checkpoint(path, mlp)
    again = LA.load_checkpoint(path)
    f = data.feats[:64]
    np.testing.assert_array_equal(LA.predict(again, f), LA.predict(mlp, f))
    mlp.close()
    again.close()
