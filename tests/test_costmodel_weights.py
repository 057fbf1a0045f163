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


def test_supernode_times_distribute_every_launch():
    """Per-supernode targets of the learned rules: each launch's time is spread over the supernodes
    of its tasks, so the per-supernode times add up to the launch times, and every fundamental
    supernode gets its final supernode's time in proportion to its share of sum c_j^2."""
    import numpy as np

    import paper_1705_06575_gb300 as S
    import workloads as w
    from paper_1705_06575_gb300 import costmodel as cm
    M = w.conduct3d(10, np.random.default_rng(4), "star")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, opt=cm.options(cm.DEFAULT), host_only=True)
    nl = s.export("factor_launches").size // 5
    ms = np.concatenate([[5.0], np.linspace(0.1, 1.0, nl)])
    t = cm.supernode_times(s, ms)
    assert t.shape == (s.info().nsuper,) and np.all(t >= 0)
    assert abs(t.sum() - ms[1:].sum()) <= 1e-9 * ms[1:].sum()
    tab = cm.fund_table(M)
    tf = cm.fund_times(tab, s, ms)
    assert tf.shape == (tab["nf"],) and abs(tf.sum() - t.sum()) <= 1e-9 * t.sum()
    X = cm.sn_features(tab, 3)
    assert X.shape == (tab["nf"], cm.NFEAT_SN) and np.isfinite(X).all()


def test_per_supernode_rules_reproduce_presets_and_oracle():
    """A rule table with every fundamental supernode on one preset gives that preset's plan; a
    random mix of rules gives the plan the oracle builds from the same rules, bit for bit."""
    import numpy as np

    import oracle
    import paper_1705_06575_gb300 as S
    import workloads as w
    from paper_1705_06575_gb300 import costmodel as cm
    M = w.dd2d9(30, np.random.default_rng(5))
    nf = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True).export("fsuper").size - 1
    for p in range(len(cm.PRESETS)):
        a = S.Solver(M.n, M.Ap, M.Ai, M.perm, opt=cm.options(p), host_only=True)
        b = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True, rules=(cm.RULES, np.full(nf, p)))
        assert np.array_equal(a.export("super"), b.export("super"))
    fr = np.random.default_rng(6).integers(0, len(cm.PRESETS), nf).astype(np.int32)
    b = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True, rules=(cm.RULES, fr))
    o = oracle.Oracle(M.n, M.Ap, M.Ai, b.export("perm"), rules=cm.RULES, fund_rule=fr, want_rel=True)
    for mine, theirs in (("super", "sn"), ("rowptr", "srp"), ("rows", "sri"), ("desc", "dk"), ("rel", "rel")):
        assert np.array_equal(b.export(mine), getattr(o, theirs)), mine
    import pytest
    with pytest.raises(S.SymError):  # one rule index per fundamental supernode is required
        S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True, rules=(cm.RULES, fr[:-1]))


def test_pretrained_per_supernode_weights_and_evaluation():
    """The packaged per-supernode networks (FP64 and mixed-precision FP32 arms) have the network
    shape, and their predictions on host features of a fresh pattern are finite per-supernode
    log times; the stored held-out evaluation covers both arms."""
    import json
    import os
    for arm in ("fp64", "fp32"):
        m = cm.pretrained_sn(arm)
        assert m.mean.shape == (cm.NFEAT_SN,) and np.all(m.std > 0)
        assert m.theta.size == ref.nparams(cm.NFEAT_SN, m.hidden) and np.all(np.isfinite(m.theta))
        tab = cm.fund_table(w.dd2d9(40, np.random.default_rng(8)))
        for p in range(len(cm.PRESETS)):
            y, _ = ref.forward(m.theta.astype(np.float64), (cm.sn_features(tab, p) - m.mean) / m.std,
                               cm.NFEAT_SN, m.hidden)
            assert y.shape == (tab["nf"],) and np.all(np.isfinite(y)) and np.all(y < np.log(1e4))
    ev = json.load(open(os.path.join(os.path.dirname(cm.__file__), "costmodel_sn_eval.json")))
    for arm in ("fp64", "fp32"):
        a = ev["arms"][arm]
        assert a["patterns"] > 0 and a["geomean_speedup_per_supernode"] > 0


def test_pretrained_pattern_fp32_weights_and_evaluation():
    """The packaged per-pattern network of the FP32 arm has the network shape, gives finite
    predictions on host features, and its stored held-out evaluation covers 400 patterns."""
    import json
    import os
    m = cm.pretrained_pattern("fp32")
    assert m.mean.shape == (cm.NFEAT,) and np.all(m.std > 0)
    assert m.theta.size == ref.nparams(cm.NFEAT, m.hidden) and np.all(np.isfinite(m.theta))
    X = cm.plan_features(w.laplace2d5(60, np.random.default_rng(1)))
    y, _ = ref.forward(m.theta.astype(np.float64), (X - m.mean) / m.std, cm.NFEAT, m.hidden)
    assert np.all(np.isfinite(y))
    ev = json.load(open(os.path.join(os.path.dirname(cm.__file__), "costmodel_pattern_fp32_eval.json")))
    assert ev["arm"] == "fp32" and ev["patterns"] == 400
