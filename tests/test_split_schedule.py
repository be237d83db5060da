"""The slab layout and halo-exchange schedule of split domains
(lbm_split_schedule, host only) on the CPU.

The schedule is run here by two gloo ranks on numpy buffers: each rank owns
slabs of a D2Q9 population field with one halo layer per cut, pull-streams
them (the data movement of Sec. II.C's stream step, halfway bounce-back at
walls, no collision) and exchanges the halo layers by send/recv exactly as
the schedule lists.  After many steps the assembled field must equal the
unsplit field streamed the same way, bit for bit, and the mass summed by an
all-reduce over the ranks must equal the whole field's.  The GPU runs the
same schedule with device copies (tests/test_gpu_split.py).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tables():
    sys.path.insert(0, ROOT)
    import oracle as O
    _, Q, c, w, _ = O.lattice_tables(O.D2Q9)
    c = np.asarray(c).reshape(Q, -1)[:, :2].astype(int)
    opp = np.array([int(np.where((c == -c[i]).all(axis=1))[0][0]) for i in range(Q)])
    return Q, c, opp


def _stream_whole(f, c, opp, per):
    """Pull f_i(y, x) <- f_i(y - cy, x - cx); across a wall the node's own
    opposite population (halfway bounce-back)."""
    Q, ny, nx = f.shape
    out = np.empty_like(f)
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    for i in range(Q):
        sy, sx = y - c[i, 1], x - c[i, 0]
        wall = np.zeros((ny, nx), bool)
        if per[1]:
            sy = sy % ny
        else:
            wall |= (sy < 0) | (sy >= ny)
        if per[0]:
            sx = sx % nx
        else:
            wall |= (sx < 0) | (sx >= nx)
        syc, sxc = np.clip(sy, 0, ny - 1), np.clip(sx, 0, nx - 1)
        out[i] = np.where(wall, f[opp[i]], f[i][syc + 0 * sxc, sxc + 0 * syc])
    return out


def _stream_slab(f, g0, n_all, c, opp, per):
    """The same on a slab [Q][n + 2][nx] (halo layers 0 and n + 1): layers
    1..n pull from the buffer without wrapping along y; a wall where the
    global source row leaves a domain not periodic in y."""
    Q, L, nx = f.shape
    n = L - 2
    out = f.copy()
    y = np.arange(1, n + 1)[:, None]
    x = np.arange(nx)[None, :]
    for i in range(Q):
        sy, sx = y - c[i, 1], x - c[i, 0]
        gy = g0 + sy - 1
        wall = np.zeros((n, nx), bool)
        if not per[1]:
            wall |= (gy < 0) | (gy >= n_all)
        if per[0]:
            sx = sx % nx
        else:
            wall |= (sx < 0) | (sx >= nx)
        syc, sxc = np.clip(sy, 0, L - 1), np.clip(sx, 0, nx - 1)
        own = f[opp[i]][1:n + 1]
        out[i][1:n + 1] = np.where(wall, own, f[i][syc + 0 * sxc, sxc + 0 * syc])
    return out


def _slab_from_whole(f, g0, n, per):
    Q, ny, nx = f.shape
    s = np.zeros((Q, n + 2, nx))
    for l in range(n + 2):
        g = g0 + l - 1
        if 0 <= g < ny or per[1]:
            s[:, l] = f[:, g % ny]
    return s


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, shape, parts, per, steps, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_2212_07494_gb300 as P
    import lbm_workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    nx, ny = shape
    Q, c, opp = _tables()
    f0 = W.SplitMix64(5).uniform(Q * ny * nx).reshape(Q, ny, nx)
    layers, copies = P.lbm_split_schedule("D2Q9", ny, parts, per[1])
    mine = [p for p in range(parts) if p % ws == rank]
    slabs = {p: _slab_from_whole(f0, layers[p][0], layers[p][1], per) for p in mine}
    for _ in range(steps):
        for p in mine:
            slabs[p] = _stream_slab(slabs[p], layers[p][0], ny, c, opp, per)
        reqs, recvs, sent = [], [], []
        for k, (dp, dl, sp, sl, i) in enumerate(copies):
            if sp in slabs and dp in slabs:
                continue
            if sp in slabs:
                sent.append(torch.from_numpy(slabs[sp][i, sl].copy()))
                reqs.append(dist.isend(sent[-1], dst=dp % ws, tag=k))
            elif dp in slabs:
                buf = torch.empty(nx, dtype=torch.float64)
                reqs.append(dist.irecv(buf, src=sp % ws, tag=k))
                recvs.append((dp, dl, i, buf))
        # copies between slabs of this rank, from the values before the exchange
        local = [(dp, dl, i, slabs[sp][i, sl].copy()) for (dp, dl, sp, sl, i) in copies
                 if sp in slabs and dp in slabs]
        for r in reqs:
            r.wait()
        for dp, dl, i, v in local:
            slabs[dp][i, dl] = v
        for dp, dl, i, buf in recvs:
            slabs[dp][i, dl] = buf.numpy()
    # mass over the owned layers, all-reduced
    m = torch.tensor([sum(float(slabs[p][:, 1:-1].sum()) for p in mine)], dtype=torch.float64)
    dist.all_reduce(m)
    owned = {p: slabs[p][:, 1:-1] for p in mine}
    out.put((rank, owned, float(m.item())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("parts,per", [(2, (1, 1)), (3, (1, 0)), (4, (0, 1)), (5, (0, 0))])
def test_two_ranks_run_the_schedule(parts, per):
    sys.path.insert(0, ROOT)
    import lbm_workloads as W
    shape, steps = (23, 17), 40
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, shape, parts, per, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nx, ny = shape
    Q, c, opp = _tables()
    f = W.SplitMix64(5).uniform(Q * ny * nx).reshape(Q, ny, nx)
    for _ in range(steps):
        f = _stream_whole(f, c, opp, per)
    import paper_2212_07494_gb300 as P
    layers, _ = P.lbm_split_schedule("D2Q9", ny, parts, per[1])
    got = np.empty_like(f)
    for _, owned, _ in res:
        for p, v in owned.items():
            g0, n = layers[p]
            got[:, g0:g0 + n] = v
    assert np.array_equal(got, f)
    for _, _, m in res:
        assert m == pytest.approx(float(f.sum()), rel=1e-12)


def test_layout_and_schedule_contents():
    """Slabs tile the axis in order; each halo gets exactly the populations
    that cross its cut (c_y = +1 from below, -1 from above), from the
    neighbour's adjacent owned layer; none across a wall."""
    sys.path.insert(0, ROOT)
    import paper_2212_07494_gb300 as P
    Q, c, opp = _tables()
    for n_all, parts, per in ((10, 3, 1), (10, 3, 0), (7, 7, 1), (5, 1, 1), (5, 1, 0)):
        layers, copies = P.lbm_split_schedule("D2Q9", n_all, parts, per)
        assert layers[0][0] == 0 and sum(n for _, n in layers) == n_all
        assert all(layers[p][0] + layers[p][1] == layers[p + 1][0] for p in range(parts - 1))
        assert max(n for _, n in layers) - min(n for _, n in layers) <= 1
        up = [i for i in range(Q) if c[i, 1] == 1]
        down = [i for i in range(Q) if c[i, 1] == -1]
        want = []
        for p in range(parts):
            n = layers[p][1]
            if p > 0 or per:
                b = (p - 1) % parts
                want += [(p, 0, b, layers[b][1], i) for i in up]
            if p < parts - 1 or per:
                a = (p + 1) % parts
                want += [(p, n + 1, a, 1, i) for i in down]
        assert copies == want
    for lat, q in (("D3Q19", 5), ("D3Q27", 9)):
        _, copies = P.lbm_split_schedule(lat, 8, 2, 1)
        assert len(copies) == 2 * 2 * q
    with pytest.raises(P.LbmError):
        P.lbm_split_schedule("D2Q9", 3, 4, 1)
