"""Serving clients in other processes (ws_server_listen): several trainer
processes with no GPU context submit requests of different env types to one
server over its Unix-domain socket, concurrently; each one's records equal
those of the same request served alone in process.  A client killed while its
request runs has the request released (its bytes return to the budget), and
the server goes on serving new clients."""
import multiprocessing as mp
import os
import time

import pytest

from paper_2408_00930_gb300 import warpsci as W
from tests.gpu_common import need_gpu
from tests.test_gpu_serving import FIELDS, GB, collect, req, slots_of

pytestmark = pytest.mark.gpu

SPECS = [("control", W.WS_ENV_CONTROL, 6000, 150, 21, False),
         ("economy", W.WS_ENV_ECONOMY, 120, 100, 22, True),
         ("landscape", W.WS_ENV_LANDSCAPE, 900, 100, 23, True),
         ("acrobot", W.WS_ENV_ACROBOT, 3000, 100, 24, False)]
DIMS = {W.WS_ENV_CONTROL: (4, 1), W.WS_ENV_ECONOMY: (16, 1), W.WS_ENV_LANDSCAPE: (24, 24),
        W.WS_ENV_ACROBOT: (6, 1)}


def _client(path, spec, out_q):
    """One trainer process: submit, then receive and acknowledge every chunk."""
    from paper_2408_00930_gb300 import serve_client
    name, env, n, h, seed, fused = spec
    c = serve_client.RemoteServer(path)
    q, _keep = req(env, n, h, seed, fused=fused)
    st, rid = c.submit(q)
    assert st == W.WS_OK, st
    chunks = []
    for ch in range(h // 50):
        assert c.wait_chunk(rid, ch, 120000) == W.WS_OK
        per = {}
        for f in FIELDS:
            st, data = c.fetch(rid, f, ch)
            assert st == W.WS_OK, (name, f, st)
            per[f] = data
        chunks.append(per)
        assert c.ack(rid, ch) == W.WS_OK
    assert c.release(rid) == W.WS_OK
    c.close()
    out_q.put((name, chunks))


def _doomed_client(path, started):
    """Submits a long request, receives its first chunk, then waits to be killed."""
    from paper_2408_00930_gb300 import serve_client
    c = serve_client.RemoteServer(path)
    q, _keep = req(W.WS_ENV_CONTROL, 60000, 1000, 99)
    st, rid = c.submit(q)
    assert st == W.WS_OK
    assert c.wait_chunk(rid, 0, 120000) == W.WS_OK
    started.set()
    time.sleep(600)


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def test_clients_in_other_processes(torch, tmp_path):
    # the same requests served alone, in process
    alone = {}
    srv = W.Server(8 * GB)
    for name, env, n, h, seed, fused in SPECS:
        q, keep = req(env, n, h, seed, fused=fused)
        st, rid = srv.submit(q)
        assert st == W.WS_OK
        alone[name] = collect(srv, rid, slots_of(q), *DIMS[env], h // 50)
        srv.release(rid)
    srv.close()

    path = os.path.join(str(tmp_path), "ws.sock")
    srv = W.Server(8 * GB)
    srv.listen(path)
    ctx = mp.get_context("spawn")
    out_q = ctx.Queue()
    started = ctx.Event()
    doomed = ctx.Process(target=_doomed_client, args=(path, started))
    doomed.start()
    assert started.wait(180)
    used_with_doomed = srv.stats()["used_bytes"]
    assert used_with_doomed > 0
    procs = [ctx.Process(target=_client, args=(path, s, out_q)) for s in SPECS]
    for p in procs:
        p.start()
    doomed.kill()                       # a client dies while its request runs
    doomed.join(30)
    got = dict(out_q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for name in alone:
        assert got[name] == alone[name], name
    # every request is gone, the killed client's included: the budget is free again
    t0 = time.time()
    while srv.stats()["used_bytes"] != 0:
        assert time.time() - t0 < 60, srv.stats()
        time.sleep(0.05)
    st = srv.stats()
    assert st["active"] == 0 and st["pending"] == 0 and st["failed"] == 0
    # the server goes on: a new client is served
    late = ctx.Process(target=_client, args=(path, SPECS[0], out_q))
    late.start()
    name, chunks = out_q.get(timeout=300)
    late.join(60)
    assert late.exitcode == 0 and chunks == alone[name]
    srv.close()
    assert not os.path.exists(path)
