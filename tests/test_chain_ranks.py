"""Algorithm 1 with the level-II chains split over ranks (the multi-GPU
design: contiguous chain blocks, the end state of a rank's last chain sent to
the next rank, an all-reduce (min) of the first failing chain index, r_star
broadcast from its owner), run as gloo ranks on CPU.

The chains of each rank are run by the FP64 oracle here (test
infrastructure), so the split run must reproduce the single-process oracle
run of Algorithm 1 exactly: the same decision log, the same accepted steps and
the same final configuration.  World sizes 2 and 3 (uneven blocks, and a last
window with fewer chains than ranks)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DG, K, P, N_STEPS = 5e-3, 3, 4, 30  # the paper's increment 1/200 (Sec. 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _glass():
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2507_20802_gb300 import synthetic as syn
    pot = oracle.make_potential(2, syn.LJ_SIGMA, syn.LJ_EPS, syn.RC_FACTOR)
    fp = oracle.make_fire(**syn.FIRE)
    x, t, H = syn.random_glass_start(64, 2, seed=23)
    q = oracle.fire(pot, fp, x, t, H)
    assert q["status"] == 0
    return pot, fp, q["x"], t, H


class _OracleChains:
    """Chains by the oracle, in the order of its own Algorithm 1: F of the
    level-I start F^(i K dgamma) r_star, then K_i sequential AQS steps; the
    equality measure is the oracle's."""

    def __init__(self, pot, fp, t):
        self.pot, self.fp, self.t = pot, fp, t

    def run(self, x_star, H_star, chains, Ki, dgamma, K_):
        import oracle
        from paper_2507_20802_gb300.chain_ranks import ChainResult
        out = []
        for i in chains:
            xs, Hs = oracle.affine_shear(x_star, H_star, i * (K_ * dgamma))
            f = oracle.fire(self.pot, self.fp, xs, self.t, Hs)
            assert f["status"] == 0
            a = oracle.aqs(self.pot, self.fp, f["x"], self.t, Hs, dgamma, Ki[i])
            assert a["status"] == 0
            out.append(ChainResult(out=f["x"], H_out=Hs, end=a["x"], H_end=a["H"], E=a["E"],
                                   tau=a["tau"], iters=a["iters"], D=a["D"]))
        return out

    def compare(self, a, b, H):
        import oracle
        return oracle.max_rel_disp(a, b, H)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2507_20802_gb300 import chain_ranks as cr
    pot, fp, x, t, H = _glass()
    r = cr.parallel_step_ranks(x, H, DG, K, P, N_STEPS, _OracleChains(pot, fp, t),
                               eq_tol=1e-6)
    q.put((rank, {k: np.asarray(v) for k, v in r.items()}))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_chain_split_over_ranks_equals_single_process(orc, world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    pot, fp, x, t, H = _glass()
    ref = orc.parallel(pot, fp, x, t, H, DG, K, P, N_STEPS, eq_tol=1e-6)
    assert ref["status"] == 0 and np.any(ref["log_eq"] == 0)  # the run has rejections
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        r = outs[rank]
        assert int(r["passes"]) == ref["iterations"]
        for k in ("log_i", "log_eq", "log_iter"):
            assert np.array_equal(r[k], ref[k]), (rank, k)
        np.testing.assert_array_equal(r["log_m"], ref["log_m"])
        for k in ("E", "tau", "iters", "D"):
            np.testing.assert_array_equal(r[k], ref[k])
        np.testing.assert_array_equal(r["x"], ref["x"])
        np.testing.assert_array_equal(r["H"], ref["H"])


def test_chain_blocks_cover_the_chains():
    sys.path.insert(0, ROOT)
    from paper_2507_20802_gb300.chain_ranks import chain_block, chain_lengths
    for P_eff in range(1, 20):
        for G in range(1, 6):
            blocks = [chain_block(P_eff, G, g) for g in range(G)]
            assert blocks[0][0] == 0 and blocks[-1][1] == P_eff
            assert all(blocks[g][1] == blocks[g + 1][0] for g in range(G - 1))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1
    assert chain_lengths(30, 3, 4) == [3, 3, 3, 3]
    assert chain_lengths(7, 3, 4) == [3, 3, 1]
    assert chain_lengths(2, 3, 4) == [2]
