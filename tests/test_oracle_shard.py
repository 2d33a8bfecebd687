"""The spatial partition of the step on CPU ranks (gloo, world sizes 2 and
4): each rank holds a slab of layers along axis 0 of the grouped spatial core
and exchanges, through the same RingExchanger the GPU shards use, the halo
layers before transport and a sum over ranks in the rounding.  The rounding
is the oracle's TT-SVD (App. A.1, the parity reference), whose QR of the
split spatial core becomes a TSQR over the ranks' R factors; the GPU shards
sum the partial left Grams of the Gram-SVD instead (checked on the GPU).  The
local arithmetic is the oracle's (test infrastructure); the sharded step must
equal the single-rank oracle step to 1e-12 at forced ranks and take the same
free rank decisions."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads
from oracle import tt
from oracle.rounding import choose_rank
from oracle.ttstep import OUTFLOW, PERIODIC, VACUUM
from oracle.ttstep import TTSN as OracleTTSN


def _problem(n, bc):
    f = workloads.random_fields(n, 9)
    return dict(n=n, L=[1.0] * len(n), n_theta=4, n_phi=8, c=1.0, a_r=1.0, dt=0.4 * min(1.0 / m for m in n),
                bc=[bc] * len(n), sigma_a=f["sigma_a"], cv=f["cv"], T0=f["T0"], eps=1e-5)


def _oracle(p, cores, T, n=None, bc=None, fields=None):
    n = n or p["n"]
    f = fields or p
    dx = [p["L"][a] / p["n"][a] for a in range(len(p["n"]))]
    return OracleTTSN(n, [dx[a] * n[a] for a in range(len(n))], p["n_theta"], p["n_phi"], p["c"], p["a_r"],
                      p["dt"], bc or p["bc"], f["sigma_a"], f["cv"], T, cores, eps=p["eps"], rounding="ttsvd")


def _sharded_round_ttsvd(cores, ex, eps, forced=None):
    """TT-SVD rounding (App. A.1) of three cores whose first core is split by
    rows over the ranks.  The QR of the split core is a TSQR: each rank's
    R factor goes into its slot of a stack that the ring's sum assembles on
    every rank, the stack's QR gives R and the rotation of each slot;
    everything else is replicated."""
    G = [np.array(c, float) for c in cores]
    world = ex.world
    # backward sweep: right-orthonormalise cores 3 and 2 (replicated); the
    # R factor of core 2 is absorbed into the split core's rows
    for k in (2, 1):
        r0, n, r1 = G[k].shape
        Q, R = np.linalg.qr(G[k].reshape(r0, n * r1).T)
        G[k] = Q.T.reshape(Q.shape[1], n, r1)
        G[k - 1] = np.tensordot(G[k - 1], R.T, axes=([2], [0]))
    nrm2 = torch.tensor([float(np.sum(G[0] ** 2))], dtype=torch.float64)
    ex.sum_(nrm2)
    delta = eps * float(np.sqrt(nrm2[0])) / np.sqrt(2.0)
    ranks = []
    # bond 0: TSQR of the split core
    _, nl, R1 = G[0].shape
    A = G[0].reshape(nl, R1)
    Qs, Rs = np.linalg.qr(A)
    k = Rs.shape[0]
    stack = np.zeros((world * R1, R1))
    stack[ex.rank * R1:ex.rank * R1 + k] = Rs
    t = torch.from_numpy(stack)
    ex.sum_(t)
    QS, R = np.linalg.qr(t.numpy())
    Qown = Qs @ QS[ex.rank * R1:ex.rank * R1 + k]
    U, S, Vt = np.linalg.svd(R, full_matrices=False)
    r = choose_rank(S, delta, None, None if forced is None else forced[0])
    ranks.append(r)
    G[0] = (Qown @ U[:, :r]).reshape(1, nl, r)
    G[1] = np.tensordot(S[:r, None] * Vt[:r], G[1], axes=([1], [0]))
    # bond 1: replicated
    r0, n, r1 = G[1].shape
    QA, RA = np.linalg.qr(G[1].reshape(r0 * n, r1))
    U, S, Vt = np.linalg.svd(RA, full_matrices=False)
    r = choose_rank(S, delta, None, None if forced is None else forced[1])
    ranks.append(r)
    G[1] = (QA @ U[:, :r]).reshape(r0, n, r)
    G[2] = np.tensordot(S[:r, None] * Vt[:r], G[2], axes=([1], [0]))
    return G, ranks


def _sharded_step(p, p0, p1, cores, T, ex, forced=None):
    """One step of the shard holding layers [p0, p1) of axis 0."""
    n = tuple(p["n"])
    plane = int(np.prod(n[1:]))
    nl = p1 - p0
    X, Th, Ph = cores
    r1 = X.shape[2]
    own = X[0].reshape(nl, plane * r1)
    send_lo, send_hi = torch.from_numpy(own[0].copy()), torch.from_numpy(own[-1].copy())
    recv_lo, recv_hi = torch.zeros_like(send_lo), torch.zeros_like(send_hi)
    ex.halo_(send_lo, send_hi, recv_lo, recv_hi)
    bc0 = p["bc"][0]
    lo, hi = recv_lo.numpy(), recv_hi.numpy()
    if p0 == 0 and bc0 != PERIODIC:
        lo = np.zeros_like(lo) if bc0 == VACUUM else own[0]
    if p1 == n[0] and bc0 != PERIODIC:
        hi = np.zeros_like(hi) if bc0 == VACUUM else own[-1]
    ext = np.concatenate([lo[None], own, hi[None]]).reshape(1, (nl + 2) * plane, r1)
    # the slab with its ghost layers: the oracle's own stencil on the interior
    # layers reads the exchanged ghosts (the ghost layers' own rows are dropped)
    sl = slice(p0 - 1, p1 + 1)
    def pad(field):
        F = field.reshape(n)
        idx = np.clip(np.arange(p0 - 1, p1 + 1), 0, n[0] - 1)
        return np.take(F, idx, axis=0).reshape(-1)
    fields = dict(sigma_a=pad(p["sigma_a"]), cv=pad(p["cv"]))
    Text = np.concatenate([np.zeros(plane), T, np.zeros(plane)])
    sub = _oracle(p, [ext, Th, Ph], Text, n=(nl + 2,) + n[1:], bc=[OUTFLOW] + list(p["bc"][1:]), fields=fields)
    grown = sub.transport(sub.cores)
    grown, E_star, _ = sub.source(grown)
    rows = slice(plane, plane + nl * plane)
    grown = [grown[0][:, rows, :], grown[1], grown[2]]
    E_star = E_star[rows]
    new, ranks = _sharded_round_ttsvd(grown, ex, p["eps"], forced)
    E_new = tt.energy_density_grouped(new, sub.g["w"], sub.g["v"], p["c"])
    cv = p["cv"].reshape(-1)[p0 * plane:p1 * plane]
    return new, T + (E_star - E_new) / cv, ranks


CASES = [((12, 9), VACUUM), ((12, 9), PERIODIC), ((8, 5, 4), OUTFLOW)]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2503_18056_gb300.shard import RingExchanger, shard_planes

        ex = RingExchanger()
        res = []
        for n, bc in CASES:
            p = _problem(n, bc)
            plane = int(np.prod(n[1:]))
            p0, p1 = shard_planes(n[0], world, rank)
            I0 = p["c"] * p["a_r"] * p["T0"].reshape(-1) ** 4 / (4 * np.pi)
            full = OracleTTSN.isotropic_cores(I0, p["n_theta"], p["n_phi"])
            for forced_run in (False, True):
                ref = _oracle(p, full, p["T0"].reshape(-1))
                cores = [full[0][:, p0 * plane:p1 * plane, :], full[1], full[2]]
                T = p["T0"].reshape(-1)[p0 * plane:p1 * plane].copy()
                ranks = []
                for m in range(3):
                    ref.step()
                    forced = list(ref.last_ranks[-1]) if forced_run else None
                    cores, T, rk = _sharded_step(p, p0, p1, cores, T, ex, forced)
                    ranks.append((rk, list(ref.last_ranks[-1])))
                Rf = ref.full().reshape(ref.nc, -1)[p0 * plane:p1 * plane]
                F = tt.full(cores).reshape(Rf.shape)
                err = float(np.linalg.norm(F - Rf) / np.linalg.norm(ref.full()))
                errT = float(np.abs(T - ref.T[p0 * plane:p1 * plane]).max())
                res.append((n, bc, forced_run, ranks, err, errT))
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_step_equals_single_rank_oracle_step(world):
    port = 30500 + 31 * world + os.getpid() % 1000
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        for n, bc, forced_run, ranks, err, errT in out[r]:
            for rk, want in ranks:
                assert list(rk) == list(want), (n, bc, forced_run, ranks)
            assert err <= 1e-12, (n, bc, forced_run, err)
            assert errT <= 1e-12, (n, bc, forced_run, errT)
