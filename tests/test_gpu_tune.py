"""Autotuner: times every fused-pass configuration on the caller's image, records
the fastest for the image's size class and TV type, and round-trips the table
through the JSON cache; the tuned default still meets the parity bar."""
import numpy as np
import pytest
import torch

import paper_2109_05496_gb300 as ctv
from paper_2109_05496_gb300 import _lib, tune
from phantoms import noisy_phantom, to_c64
from tests.helpers import oracle_constraint, run_oracle
from tests.test_gpu_denoise import check_parity

pytestmark = pytest.mark.gpu


def test_autotune_records_and_roundtrips(tmp_path, monkeypatch):
    lib = _lib.load()
    m, n = 200, 300
    _, noisy = noisy_phantom(m, n, 0.1, seed=31)
    b = torch.from_numpy(to_c64(noisy)).cuda()
    res = tune.autotune(b, 0.05, "tv2_iso", 30, ctv.Constraint(amp_max=1.0), repeats=1)
    ncfg = lib.ctv_num_configs()
    assert 0 <= res["best"] < ncfg
    assert all(t > 0 for t in res["times_ms"])
    assert res["best"] == int(np.argmin(res["times_ms"]))
    sc = lib.ctv_size_class(m, n)
    assert sc == int(np.floor(np.log2(m * n)))
    assert tune.table()["%d/2" % sc] == res["best"]
    # the tuned default solves within the parity bar
    x = ctv.denoise(b, 0.05, "tv2_iso", 30, ctv.Constraint(amp_max=1.0))
    torch.cuda.synchronize()
    bp, ores = run_oracle(noisy, 0.05, 30, "tv2_iso", 0.5, oracle_constraint(1.0))
    check_parity(x.cpu().numpy(), ores, bp, noisy, 0.05, "tv2_iso", 0.5)
    # JSON round trip
    path = str(tmp_path / "tune.json")
    tune.save(path)
    _lib.check("ctv_tune_set", lib.ctv_tune_set(sc, 2, -1))
    assert "%d/2" % sc not in tune.table()
    assert tune.load(path) >= 1
    assert tune.table()["%d/2" % sc] == res["best"]
    _lib.check("ctv_tune_set", lib.ctv_tune_set(sc, 2, -1))
