"""Autotuner: selection and cache logic on CPU (fake timings); device tuning on the GPU gives
options whose results equal the defaults'."""
import json

import numpy as np
import pytest
import torch

from paper_2410_22764_gb300 import autotune


def test_choose_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    cands = [{"ctas": 152}, {"ctas": 304}, {"ctas": 608}]
    fake = {152: 3.0, 304: 1.5, 608: 2.0}
    calls = []

    def measure(c):
        calls.append(c)
        return fake[c["ctas"]]
    best, timings = autotune.choose("gpu|single|x", cands, measure, path)
    assert best == {"ctas": 304} and len(calls) == 3 and len(timings) == 3
    best2, _ = autotune.choose("gpu|single|x", cands, lambda c: 1 / 0, path)   # from the cache
    assert best2 == best
    fake[608] = 0.5
    best3, _ = autotune.choose("gpu|single|x", cands, measure, path, retune=True)
    assert best3 == {"ctas": 608}
    assert json.load(open(path))["gpu|single|x"]["best"] == {"ctas": 608}


def test_keys_bucket_similar_shapes():
    assert autotune.single_key("G", 1_000_000, 4, False) == autotune.single_key("G", 1_100_000, 4,
                                                                                 False)
    assert autotune.single_key("G", 1000, 4, False) != autotune.single_key("G", 1000, 4, True)
    assert autotune.batch_key("G", [100] * 10, [2] * 10, False).startswith("G|batch|count2^3")


@pytest.mark.gpu
def test_tuned_options_give_default_results(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22764_gb300 import dfamin, inputs as I
    path = str(tmp_path / "tune.json")
    d = I.inflated_dfa(20000, 4, 5, 0.5, 4)[0]
    dd, aa = dfamin.to_device(d.delta, d.accept)
    opt, timings = autotune.tune_single(d.n, d.k, dd, aa, path=path)
    assert len(timings) >= 4
    a = dfamin.minimize_ex(d.n, d.k, dd, aa, opt=opt).host()
    b = dfamin.minimize_ex(d.n, d.k, dd, aa).host()
    assert np.array_equal(a[0], b[0]) and a[1:] == b[1:]
    ns, ks, ps, seeds = I.batch_sizes(200, 2, n_hi=50000)
    delta, acc, so, kk = I.random_batch(ns, ks, ps, seeds)
    dd = torch.from_numpy(delta).cuda()
    aa = torch.from_numpy(acc.view(np.int32)).cuda()
    bopt, bt = autotune.tune_batch(so, kk, dd, aa, path=path)
    assert len(bt) >= 9
    tuned, default = dfamin.BatchPlan(so, kk, bopt), dfamin.BatchPlan(so, kk)
    o1, p1 = tuned.run(dd, aa)
    o2, p2 = default.run(dd, aa)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2) and torch.equal(p1, p2)


def test_leader_candidates_only_when_allowed():
    plain = autotune.single_candidates(100000, 152)
    both = autotune.single_candidates(100000, 152, leader=True)
    assert not any("algorithm" in c for c in plain)
    assert {json.dumps(c, sort_keys=True) for c in plain} < {json.dumps(c, sort_keys=True)
                                                              for c in both}
    assert all(c.get("algorithm") == 1 for c in both if c not in plain)
    assert autotune.single_key("G", 10**5, 4, False, True) != autotune.single_key("G", 10**5, 4,
                                                                                   False)


@pytest.mark.gpu
def test_tuner_may_pick_the_leader_election(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22764_gb300 import dfamin, inputs as I
    d = I.bitsplitter_dfa(14)
    dd, aa = dfamin.to_device(d.delta, d.accept)
    opt, timings = autotune.tune_single(d.n, d.k, dd, aa, path=str(tmp_path / "t.json"),
                                        allow_leader=True)
    assert any('"algorithm": 1' in key for key in timings)
    got = dfamin.minimize_ex(d.n, d.k, dd, aa, opt=opt).host()
    want = dfamin.minimize_ex(d.n, d.k, dd, aa).host()
    assert np.array_equal(got[0], want[0]) and got[1] == want[1] and got[3] == 0
