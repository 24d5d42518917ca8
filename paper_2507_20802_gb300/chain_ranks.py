"""Algorithm 1 with its level-II chains split over ranks (one GPU per rank).

The P chains of a pass are independent until the equality tests (Sec. 3.3,
Eq. 19), so rank g of G takes a contiguous block of chains.  One pass needs
three exchanges, and nothing else crosses ranks:

1. point to point: the end state of the last chain of rank g goes to rank
   g + 1, whose first chain's equality test (Sec. 3.4, Eq. 20) compares it
   with its own first minimum;
2. an all-reduce (minimum) of the first failing chain index over the ranks
   (Algorithm 1's decision: the first unequal pair ends the accepted range);
3. a broadcast of r_star (the end of the last accepted chain, and its cell)
   from the rank that owns that chain.

The per-step records of the accepted chains (energy, stress, FIRE iterations,
non-affine displacement) and the decision log are gathered to every rank as
small Python objects.

The chains of a rank are run, and the equality measure is evaluated, by a
``chains`` object (methods ``run`` and ``compare``), so the exchange logic
does not depend on where the chains run: ``LibraryChains`` runs both with the
CUDA library on this rank's GPU.  This module does none of the method's
arithmetic itself.  Every rank starts from rank 0's r_star and cell
(broadcast once at the start).

Readings of Algorithm 1 (as in the single-process library): the last window
runs P_eff = min(P, ceil(rem / K)) chains and the last one is shortened to
end exactly at n_steps; on a failed test at chain i, r_star <- end of chain
i - 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ChainResult:
    """One level-II chain: F applied to the level-I start (``out``, at the
    strain i K dgamma, cell ``H_out``), then K_i fine AQS steps (``end``, cell
    ``H_end``) with their per-step records."""
    out: np.ndarray
    H_out: np.ndarray
    end: np.ndarray
    H_end: np.ndarray
    E: np.ndarray
    tau: np.ndarray
    iters: np.ndarray
    D: np.ndarray


@dataclass
class PassLog:
    """Decisions of one pass: the tests made up to the first failure."""
    chain: list = field(default_factory=list)
    equal: list = field(default_factory=list)
    m: list = field(default_factory=list)


def chain_block(P_eff: int, G: int, g: int) -> tuple[int, int]:
    """Contiguous chains [lo, hi) of rank g; the first P_eff mod G ranks take
    one chain more."""
    base, extra = divmod(P_eff, G)
    lo = g * base + min(g, extra)
    return lo, lo + base + (1 if g < extra else 0)


def chain_lengths(rem: int, K: int, P: int) -> list[int]:
    P_eff = min(P, -(-rem // K))
    Ki = [K] * P_eff
    if rem < P_eff * K:
        Ki[-1] = rem - (P_eff - 1) * K
    return Ki


def _owner(i: int, P_eff: int, G: int) -> int:
    for g in range(G):
        lo, hi = chain_block(P_eff, G, g)
        if lo <= i < hi:
            return g
    raise ValueError(i)


def parallel_step_ranks(x_star, H_star, dgamma, K, P, n_steps, chains, eq_tol=1e-6,
                        group=None, device="cpu"):
    """Algorithm 1 from the minimum x_star (cell H_star) with the chains split
    over the ranks of ``group`` (torch.distributed, already initialised).
    Every rank calls it; every rank returns the same dict: the final r_star
    and cell, per accepted step E, tau, FIRE iterations and D, the decision
    log and the number of passes."""
    import torch
    import torch.distributed as dist

    G, g = dist.get_world_size(group), dist.get_rank(group)
    x = torch.tensor(np.asarray(x_star, dtype=np.float64), device=device)
    H = torch.tensor(np.asarray(H_star, dtype=np.float64), device=device)
    dist.broadcast(x, src=0, group=group)  # every rank starts from rank 0's r_star
    dist.broadcast(H, src=0, group=group)
    E, tau, iters, D = [], [], [], []
    logs = []
    n_cur, passes = 0, 0
    while n_cur < n_steps:
        Ki = chain_lengths(n_steps - n_cur, K, P)
        P_eff = len(Ki)
        lo, hi = chain_block(P_eff, G, g)
        xs, Hs = x.cpu().numpy(), H.cpu().numpy()
        local = chains.run(xs, Hs, list(range(lo, hi)), Ki, dgamma, K) if hi > lo else []
        # 1. end of the last chain of rank g -> rank g + 1 (ranks with chains only)
        prev_end = None
        if hi > lo and g + 1 < G and chain_block(P_eff, G, g + 1)[1] > hi:
            dist.send(torch.tensor(local[-1].end, device=device), dst=g + 1, group=group)
        if hi > lo and lo > 0:
            buf = torch.empty_like(x)
            dist.recv(buf, src=g - 1, group=group)
            prev_end = buf.cpu().numpy()
        # local equality tests i = lo..hi-1 (i >= 1): incoming = end of chain
        # i - 1, outgoing = first minimum of chain i, both at strain i K dgamma
        tests = []
        for k, i in enumerate(range(lo, hi)):
            if i == 0:
                continue
            inc = prev_end if k == 0 else local[k - 1].end
            m = chains.compare(inc, local[k].out, local[k].H_out)
            tests.append((i, m < eq_tol, m))
        first_local = next((i for i, eq, _ in tests if not eq), P_eff)
        # 2. first failing chain over all ranks
        ff = torch.tensor([first_local], dtype=torch.int64, device=device)
        dist.all_reduce(ff, op=dist.ReduceOp.MIN, group=group)
        first_fail = int(ff.item())
        last = P_eff - 1 if first_fail >= P_eff else first_fail - 1
        # records of accepted chains and the tests, gathered as objects
        mine = {"tests": tests,
                "rec": {i: (r.E, r.tau, r.iters, r.D) for i, r in zip(range(lo, hi), local)
                        if i <= last}}
        allr = [None] * G
        dist.all_gather_object(allr, mine, group=group)
        all_tests = sorted(t for a in allr for t in a["tests"])
        log = PassLog()
        for i, eq, m in all_tests:
            log.chain.append(i)
            log.equal.append(bool(eq))
            log.m.append(m)
            if not eq:
                break
        logs.append(log)
        recs = {}
        for a in allr:
            recs.update(a["rec"])
        for i in range(last + 1):
            e, t_, it, d = recs[i]
            E.extend(e); tau.extend(t_); iters.extend(it); D.extend(d)
        # 3. r_star <- end of chain `last`, broadcast from its owner
        own = _owner(last, P_eff, G)
        if g == own:
            r = local[last - lo]
            x = torch.tensor(r.end, device=device)
            H = torch.tensor(r.H_end, device=device)
        dist.broadcast(x, src=own, group=group)
        dist.broadcast(H, src=own, group=group)
        n_cur += sum(Ki[:last + 1])
        passes += 1
    return {"x": x.cpu().numpy(), "H": H.cpu().numpy(), "E": np.array(E), "tau": np.array(tau),
            "iters": np.array(iters), "D": np.array(D), "passes": passes,
            "log_i": np.array([i for lg in logs for i in lg.chain], dtype=np.int32),
            "log_eq": np.array([e for lg in logs for e in lg.equal], dtype=np.uint8),
            "log_m": np.array([m for lg in logs for m in lg.m]),
            "log_iter": np.array([p for p, lg in enumerate(logs) for _ in lg.chain],
                                 dtype=np.int64)}


class LibraryChains:
    """Runs this rank's chains with the CUDA library on the current GPU:
    level I (Eq. 18) by aqs_affine_shear of per-chain copies of r_star, each
    chain's first minimisation by aqs_minimize and its K_i fine steps by
    aqs_run_sequential (one system per chain length); the equality measure
    by aqs_compare_configs on a two-replica system."""

    def __init__(self, types, sigma, eps, rc_factor=2.5, precision=None, fire=None):
        from . import aqs as A
        self.A = A
        self.types = np.ascontiguousarray(types, dtype=np.int32)
        self.sigma, self.eps, self.rc = sigma, eps, rc_factor
        self.prec = A.AQS_MIXED if precision is None else precision
        self.fire = fire
        self.cmp = None

    def run(self, x_star, H_star, chains, Ki, dgamma, K):
        A = self.A
        res = {}
        for L in sorted({Ki[i] for i in chains}):
            grp = [i for i in chains if Ki[i] == L]
            R, n = len(grp), len(x_star)
            s = A.System(np.tile(x_star, (R, 1)), np.tile(self.types, R),
                         np.tile(H_star[None], (R, 1, 1)), [n] * R, self.sigma, self.eps,
                         self.rc, precision=self.prec)
            s.shear(np.array([i * K * dgamma for i in grp]))
            s.minimize(self.fire)
            outs = [(s.positions(r), s.box(r)) for r in range(R)]
            o = s.run_sequential(dgamma, L, self.fire)
            for r, i in enumerate(grp):
                res[i] = ChainResult(out=outs[r][0], H_out=outs[r][1], end=s.positions(r),
                                     H_end=s.box(r), E=o["E"][:, r], tau=o["tau"][:, r],
                                     iters=o["iters"][:, r], D=o["D"][:, r])
            s.close()
        return [res[i] for i in chains]

    def compare(self, a, b, H):
        A = self.A
        if self.cmp is None or self.cmp.n_atoms[0] != len(a):
            self.cmp = A.System(np.concatenate([a, b]), np.tile(self.types, 2),
                                np.stack([H, H]), [len(a)] * 2, self.sigma, self.eps, self.rc,
                                precision=A.AQS_FP64)
        else:
            for r, pos in enumerate((a, b)):
                A.aqs_set_box(self.cmp.h, r, H)
                self.cmp.set_positions(np.ascontiguousarray(pos, dtype=np.float64), r)
        m, _ = A.aqs_compare_configs(self.cmp.h, 0, self.cmp.h, 1, 1.0)
        return m
