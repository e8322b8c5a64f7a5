"""Host-side logic of the warm-start training module and the shipped parameters (no GPU):
the disjoint union used for minibatches, the parameter layout shared by the library, the
oracle and the initialiser, and the shipped parameters with their training record."""
import json
import os

import numpy as np
import pytest

from oracle import mpnn as omp


@pytest.fixture(scope="module")
def ws():
    from paper_2307_15969_gb300 import build
    build.build()
    from paper_2307_15969_gb300 import warmstart
    return warmstart


def test_parameter_count_agrees_everywhere(ws):
    from paper_2307_15969_gb300 import lowd
    P = lowd.lowd_mpnn_param_count()
    assert P == omp.param_count() == ws.init_params(0).shape[0] == 25088


def test_union_is_a_disjoint_union(ws):
    a = dict(n=3, lo=np.array([0, 1], np.int32), hi=np.array([1, 2], np.int32), t=np.array([1, 2, 3], np.float32))
    b = dict(n=2, lo=np.array([0], np.int32), hi=np.array([1], np.int32), t=np.array([4, 5], np.float32))
    n, lo, hi, t = ws.union([a, b])
    assert n == 5
    assert lo.tolist() == [0, 1, 3] and hi.tolist() == [1, 2, 4]
    assert t.tolist() == [1, 2, 3, 4, 5]


def test_initialiser_starts_near_the_equal_split(ws):
    p = ws.init_params(3)
    W_in, b_in, Ws, bs, q = omp.unpack(p)
    assert np.all(b_in == 0) and all(np.all(b == 0) for b in bs)
    assert np.abs(q).max() <= 0.01
    assert np.abs(W_in).max() <= np.sqrt(2.0) and all(np.abs(W).max() <= np.sqrt(6 / 128) for W in Ws)


def test_shipped_parameters_and_record(ws):
    p = ws.load_params()
    assert p.dtype == np.float32 and np.all(np.isfinite(p))
    rec = json.load(open(os.path.join(os.path.dirname(ws.PARAMS_PATH), "warmstart_record.json")))
    assert rec["graphs"] == 20000 and rec["cores"] > 0
    assert rec["best_val_loss"] < 0.05 * rec["equal_split_val_loss"]
    # the shipped network is not the equal split: its readout is nonzero
    assert np.abs(omp.unpack(p)[4]).max() > 0
