"""Multi-process shot sharding on CPU: world_size-2 gloo ranks, each running the FP64 oracle on
its shots, all-reduce the misfit and gradient; the result equals the single-process gradient.
Also a rank that fails before the collective makes the other rank's collective end with an
error within a short process-group timeout (failure detection on the host)."""
import datetime
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1804_01184_gb300 import inputs as I
from paper_1804_01184_gb300.dist import shot_range


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def case():
    w = I.small_case(seed=70, nx=30, nz=26, nt=80, ns=5, nr=6, sponge=4, pz=I.PZ_IP_RHO)
    g = oracle.make_grid(**w.grid_kwargs())
    data = oracle.model(g, w.pz, w.xi_a * 1.3, w.xi_b * 0.8, w.src_xy, w.wavelet, w.rec_xy)
    return w, g, data


def fcase():
    from oracle import fborn as FB
    w = I.small_freq_case(seed=71, nx=11, nz=9, ns=3, nr=5, nf=5, pz=I.PZ_VP_IP)
    fg = FB.FGrid(**w.fgrid_kwargs())
    q = FB.model(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, w.pz, 1.2 * w.xi_a, 0.7 * w.xi_b, FB.NONLINEAR)
    return w, fg, q


def fworker(rank, world, port, out):
    import torch.distributed as dist

    from oracle import fborn as FB
    from paper_1804_01184_gb300.dist import sharded_frequency_gradient
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    w, fg, q = fcase()
    try:
        def local(fr, sp, d):
            if len(fr) == 0:
                return 0.0, np.zeros((2, w.nz, w.nx))
            J, ga, gb = FB.gradient(fg, fr, sp, w.src_xy, w.rec_xy, w.pz, w.xi_a, w.xi_b, d, FB.LINEAR)
            return J, np.stack([ga, gb])

        J, G = sharded_frequency_gradient(local, w.freqs, w.spectrum, q)
        out.put((rank, "ok", J, G.numpy()))
    except Exception as e:   # noqa: BLE001 - reported to the parent
        out.put((rank, "error", repr(e), None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:   # noqa: BLE001
            pass


def worker(rank, world, port, out, fail_rank):
    import torch
    import torch.distributed as dist

    from paper_1804_01184_gb300.dist import sharded_gradient
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    w, g, data = case()
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure before the collective")

        def local(src, d):
            if src.shape[0] == 0:
                return 0.0, np.zeros((5, 2, w.nz, w.nx))
            return oracle.gradient(g, w.pz, w.xi_a * 0.5, w.xi_b * 0.5, src, w.wavelet, w.rec_xy, d)

        J, G = sharded_gradient(local, w.src_xy, data)
        out.put((rank, "ok", J, G.numpy()))
    except Exception as e:   # noqa: BLE001 - reported to the parent
        out.put((rank, "error", repr(e), None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:   # noqa: BLE001
            pass


def run(world, fail_rank=-1, target=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) if target else
             ctx.Process(target=worker, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    return sorted(res, key=lambda r: r[0])


def test_shot_range_partitions():
    for ns in (0, 1, 5, 64):
        for world in (1, 2, 3, 8):
            rs = [shot_range(ns, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == ns
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(h - l for l, h in rs) - min(h - l for l, h in rs) <= 1


def test_sharded_gradient_equals_single_process():
    w, g, data = case()
    J, G = oracle.gradient(g, w.pz, w.xi_a * 0.5, w.xi_b * 0.5, w.src_xy, w.wavelet, w.rec_xy, data)
    res = run(2)
    for rank, status, Jr, Gr in res:
        assert status == "ok", Jr
        assert abs(Jr - J) <= 1e-12 * J
        np.testing.assert_allclose(Gr, G, rtol=1e-12, atol=1e-12 * np.abs(G).max())


def test_failed_rank_is_detected():
    res = run(2, fail_rank=1)
    assert res[1][1] == "error" and "injected" in res[1][2]
    assert res[0][1] == "error"      # the surviving rank's all-reduce fails (peer gone / timeout)


def test_frequency_sharded_born_gradient_equals_single_process():
    """Schemes I/II: two gloo ranks each take half of the frequencies (the FP64 frequency-domain
    oracle on its part); the all-reduced misfit and gradient equal the single-process ones."""
    from oracle import fborn as FB
    w, fg, q = fcase()
    J, ga, gb = FB.gradient(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, w.pz, w.xi_a, w.xi_b, q, FB.LINEAR)
    G = np.stack([ga, gb])
    for rank, status, Jr, Gr in run(2, target=fworker):
        assert status == "ok", Jr
        assert abs(Jr - J) <= 1e-12 * J
        np.testing.assert_allclose(Gr, G, rtol=1e-10, atol=1e-12 * np.abs(G).max())
