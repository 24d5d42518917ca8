"""The library-backed chain runner of the multi-rank Algorithm 1
(chain_ranks.LibraryChains) on the GPU, as a single gloo rank: chains run by
the CUDA library, equality measured by aqs_compare_configs, and the stored
oracle run of Algorithm 1 (N = 256 glass, dgamma = 1/200, K = 3, P = 4, 30
steps) reproduced: decision log, energies (1e-9), events, final positions."""
import os
import socket

import numpy as np
import pytest

from conftest import load_golden

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_library_chains_reproduce_the_golden_decisions(syn):
    torch = pytest.importorskip("torch")
    import torch.distributed as dist
    from paper_2507_20802_gb300 import aqs as A, chain_ranks as cr
    g = load_golden("glass_2d_n256_s0.npz")
    gold = load_golden("par_2d_n256_s0.npz")
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        ch = cr.LibraryChains(g["types"], syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR,
                              precision=A.AQS_FP64)
        r = cr.parallel_step_ranks(g["x"], g["H"], float(gold["dgamma"]), int(gold["K"]),
                                   int(gold["P"]), int(gold["n_steps"]), ch,
                                   eq_tol=float(gold["eq_tol"]))
    finally:
        dist.destroy_process_group()
    assert np.array_equal(r["log_i"], gold["log_i"])
    assert np.array_equal(r["log_eq"], gold["log_eq"])
    assert int(r["passes"]) == int(gold["iterations"])
    np.testing.assert_allclose(r["E"], gold["E"], rtol=1e-9)
    assert np.array_equal(r["D"] > 1e-2, gold["D"] > 1e-2)
    d = r["x"] - gold["x"]
    H = gold["H"]
    for c in (1, 0):
        d -= np.round(d[:, c] / H[c, c])[:, None] * H[:, c][None, :]
    d -= d.mean(axis=0)
    assert np.sqrt((d * d).sum(1)).max() < 1e-6
