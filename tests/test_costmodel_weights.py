"""The packaged cost-model weights: shape, normalisation and host-side use (no GPU). The network
is evaluated here with the FP64 reference MLP on features from host-only inspections."""
import numpy as np

import workloads as w
from oracle import mlp as ref
from paper_1705_06575_gb300 import costmodel as cm


def test_pretrained_weights_have_the_network_shape():
    m = cm.pretrained()
    assert m.hidden == cm.HIDDEN
    assert m.mean.shape == (cm.NFEAT,) and m.std.shape == (cm.NFEAT,)
    assert np.all(m.std > 0)
    assert m.theta.size == ref.nparams(cm.NFEAT, cm.HIDDEN)
    assert np.all(np.isfinite(m.theta))


def test_pretrained_choice_on_host_features():
    """Predicted log times are finite and of the order of the training targets (log ms of
    factorizations between ~0.5 ms and a few seconds); the choice is a valid preset."""
    m = cm.pretrained()
    for M in (w.laplace2d5(60, np.random.default_rng(1)), w.conduct3d(14, np.random.default_rng(2), "star")):
        X = cm.plan_features(M)
        assert X.shape == (len(cm.PRESETS), cm.NFEAT)
        y, _ = ref.forward(m.theta.astype(np.float64), (X - m.mean) / m.std, cm.NFEAT, cm.HIDDEN)
        assert np.all(np.isfinite(y))
        assert np.all((y > np.log(0.05)) & (y < np.log(1e5)))
        assert 0 <= int(np.argmin(y)) < len(cm.PRESETS)
