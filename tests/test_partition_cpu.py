"""The weighted partition's host side (imga_partition_* on a host-only mesh, no GPU) and its halo
exchange between two gloo ranks on CPU (the exchange step of a multi-GPU residual / J v).

* The k element ranges tile the Morton order; every node has one owner; a part's ghosts are the
  nodes its elements touch through M_e (corners and hanging parents) that another part owns.
* Two gloo ranks, one part each: owned rows in, ghost rows filled by send / receive of the halo
  lists, then a reduce-add of per-element contributions (the partial rows of ghosts sent back to
  their owners): every owned row equals the sum over all elements, as on one rank.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2009_00706_gb300 import api  # noqa: E402
from paper_2009_00706_gb300 import inputs as I  # noqa: E402


def _mesh():
    reg = [I.Region(I.REGION_SPHERE_BAND, 5, (0.45, 0.5, 0.55, 0.2, 0.04))]
    return api.Mesh((0, 0, 0), (1, 1, 1), 3, reg, None, 2, device=-1)


def _touch(ex, n_nodes, e):
    """(node, weight) pairs element e reaches through M_e"""
    out = []
    for c in range(8):
        idx = int(ex["conn"][e, c])
        if idx < n_nodes:
            out.append((idx, 1.0))
        else:
            h = idx - n_nodes
            k = int(ex["hang_np"][h])
            out += [(int(ex["hang_parents"][h, q]), 1.0 / k) for q in range(k)]
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 7])
def test_partition_tiles_elements_and_nodes(k):
    m = _mesh()
    ex = m.export()
    P = api.Partition(m, k)
    assert P.k == k
    assert P.elem_off[0] == 0 and P.elem_off[-1] == m.n_elem and np.all(np.diff(P.elem_off) >= 1)
    # unit weights on a host-only mesh: balanced to one element
    assert np.abs(P.weight - m.n_elem / k).max() <= 1.0 + 1e-9
    owner = -np.ones(m.n_nodes, np.int64)
    for p in range(k):
        nodes, gown = P.nodes(p)
        own, ghost = nodes[: P.n_owned[p]], nodes[P.n_owned[p]:]
        assert np.all(owner[own] == -1)
        owner[own] = p
        touched = set()
        for e in range(P.elem_off[p], P.elem_off[p + 1]):
            touched.update(n for n, _ in _touch(ex, m.n_nodes, e))
        assert set(nodes.tolist()) == touched
        assert np.all(gown < p) and np.all(gown != p)        # the lowest touching part owns
        assert np.all(np.diff(own) > 0) and np.all(np.diff(ghost) > 0)
    assert np.all(owner >= 0)
    for p in range(k):
        nodes, gown = P.nodes(p)
        assert np.array_equal(owner[nodes[P.n_owned[p]:]], gown)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = _mesh()
        ex = m.export()
        P = api.Partition(m, world)
        nodes, gown = P.nodes(rank)
        no = int(P.n_owned[rank])
        glob = I.normal(5, 4 * m.n_nodes).reshape(-1, 4)
        # 1. owned rows in; 2. halo gather: every part sends the owned rows its neighbours hold as ghosts
        local = np.zeros((nodes.size, 4))
        local[:no] = glob[nodes[:no]]
        g2l = {int(n): i for i, n in enumerate(nodes)}
        lists = [P.nodes(p) for p in range(world)]
        for other in range(world):
            if other == rank:
                continue
            onodes, oown = lists[other]
            ono = int(P.n_owned[other])
            wanted = onodes[ono:][oown == rank]                  # my owned rows `other` keeps as ghosts
            mine = nodes[no:][gown == other]                     # my ghosts `other` owns
            sendbuf = torch.from_numpy(np.ascontiguousarray(local[[g2l[int(n)] for n in wanted]]))
            recvbuf = torch.zeros((mine.size, 4), dtype=torch.float64)
            reqs = [dist.isend(sendbuf, other), dist.irecv(recvbuf, other)]
            for r in reqs:
                r.wait()
            local[[g2l[int(n)] for n in mine]] = recvbuf.numpy()
        ghost_ok = bool(np.array_equal(local, glob[nodes]))
        # 3. per-element contributions of my elements; 4. reduce-add of the ghost partial rows
        part = np.zeros((nodes.size, 4))
        for e in range(P.elem_off[rank], P.elem_off[rank + 1]):
            for n, w in _touch(ex, m.n_nodes, e):
                part[g2l[n]] += w * (1.0 + e) * np.arange(1, 5)
        for other in range(world):
            if other == rank:
                continue
            onodes, oown = lists[other]
            ono = int(P.n_owned[other])
            mine = nodes[no:][gown == other]
            theirs = onodes[ono:][oown == rank]
            sendbuf = torch.from_numpy(np.ascontiguousarray(part[[g2l[int(n)] for n in mine]]))
            recvbuf = torch.zeros((theirs.size, 4), dtype=torch.float64)
            reqs = [dist.isend(sendbuf, other), dist.irecv(recvbuf, other)]
            for r in reqs:
                r.wait()
            part[[g2l[int(n)] for n in theirs]] += recvbuf.numpy()
        # the same sums on one rank
        full = np.zeros((m.n_nodes, 4))
        for e in range(m.n_elem):
            for n, w in _touch(ex, m.n_nodes, e):
                full[n] += w * (1.0 + e) * np.arange(1, 5)
        reduce_err = float(np.abs(part[:no] - full[nodes[:no]]).max() / np.abs(full).max())
        q.put((rank, ghost_ok, reduce_err, int(nodes.size - no)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_halo_gather_and_reduce_add():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ghost_ok, reduce_err, n_ghost in res:
        assert ghost_ok
        assert reduce_err <= 1e-14
    assert res[1][3] > 0          # the second part has a ghost layer
