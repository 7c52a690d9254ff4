"""Serving runtime: sessions with device-resident state, continuously batched.

Each result must be the same whether the request ran alone (its own
dpvo_ba_solve) or packed into a batch with other sessions' requests, within
the solve tolerance; sessions are admitted by the memory budget.
"""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from tests.gpu_util import TOL_DEPTH, TOL_POSE, err, err_update

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _alone(scene, poses, patches, target, weight):
    """The same request solved by itself through dpvo_ba_solve."""
    sc = dataclasses.replace(scene, poses=poses, patches=patches, target=target, weight=weight)
    s = ba.Solver()
    p = ba.problem_from_scene(sc)
    s.solve([p])
    torch.cuda.synchronize()
    out = p.poses.cpu().numpy(), p.patches.cpu().numpy(), int(p.status.item())
    s.close()
    return out


def test_results_alone_equal_results_in_the_mix():
    _need_gpu()
    rng = np.random.default_rng(0)
    scenes = S.make_serving_mix(10, base_seed=7)
    srv = ba.Solver()
    srv.serve_start(32, 3072, 66000, 2, max_batch=16, max_in_flight=2)
    try:
        sids = [srv.session_open(sc) for sc in scenes]
        state = [(sc.poses.copy(), sc.patches.copy()) for sc in scenes]
        for rnd in range(2):
            reqs = [S.refresh_factors(sc, 100 * rnd + b) for b, sc in enumerate(scenes)]
            tickets = [srv.submit(sid, r.target, r.weight) for sid, r in zip(sids, reqs)]
            for tk in tickets:
                st, lat = srv.wait(tk, 20000)
                assert st == 0 and lat > 0
            for b, (sc, sid, r) in enumerate(zip(scenes, sids, reqs)):
                poses, patches = srv.session_read(sid, sc.n_frames, sc.n_patches)
                ap, apt, ast = _alone(sc, state[b][0], state[b][1], r.target, r.weight)
                assert ast == 0
                t0 = sc.t0
                assert err_update(poses[t0:], ap[t0:], state[b][0][t0:], TOL_POSE) < TOL_POSE
                assert err_update(patches[:, 2], apt[:, 2], state[b][1][:, 2], TOL_DEPTH) < TOL_DEPTH
                state[b] = (poses, patches)
        for sid in sids:
            srv.session_close(sid)
    finally:
        srv.serve_stop()
        srv.close()


def test_sessions_are_admitted_by_the_memory_budget():
    _need_gpu()
    sc = S.make_scene(S.WINDOW_N22, 3)
    one = 1_200_000        # a 22-frame, 2112-patch, 39,552-edge session holds ~1.1 MB
    srv = ba.Solver(mem_budget_bytes=3 * one)
    srv.serve_start(22, 2112, 39552, 2, max_batch=4, max_in_flight=1)
    try:
        a = [srv.session_open(sc) for _ in range(3)]
        with pytest.raises(ba.BAError) as e:
            srv.session_open(sc)
        assert e.value.code == ba.EBUSY
        srv.session_close(a[0])
        b = srv.session_open(sc)
        tk = srv.submit(b, sc.target, sc.weight)
        st, _ = srv.wait(tk)
        assert st == 0
    finally:
        srv.serve_stop()
        srv.close()


def test_one_request_per_session_and_unknown_tickets():
    _need_gpu()
    sc = S.make_scene(S.PLAIN_N8, 4)
    srv = ba.Solver()
    srv.serve_start(8, 512, 4096, 2, max_batch=4, max_in_flight=1)
    try:
        sid = srv.session_open(sc)
        tk = srv.submit(sid, sc.target, sc.weight)
        try:
            tk2 = srv.submit(sid, sc.target, sc.weight)
        except ba.BAError as err:
            assert err.code == ba.EBUSY
        else:           # the first request may already have finished
            srv.wait(tk2)
        srv.wait(tk)
        with pytest.raises(ba.BAError) as e:
            srv.wait(tk)                  # collected already
        assert e.value.code == ba.ENOTFOUND
        with pytest.raises(ba.BAError) as e:
            srv.submit(12345, sc.target, sc.weight)
        assert e.value.code == ba.ENOTFOUND
    finally:
        srv.serve_stop()
        srv.close()


def test_sliding_window_sessions_equal_the_same_window_alone():
    """Window sessions (the paper's Default and Fast shapes: 96 patches / 10
    free poses and 48 / 7, radius 13, 22-frame windows) served together with
    fixed-graph sessions.  Every request appends a frame (pixel centres, edge
    revisions and weights from the client) and solves the window.  After each
    frame, each session's state must equal the same frame appended to a window
    of its own (dpvo_ba_window_append) and solved alone (dpvo_ba_solve).  The
    reference window is reset to the served state before each frame, so every
    comparison covers one append and one solve; 24 frames exercise the
    dropping of the oldest frame once the window is full."""
    _need_gpu()
    rng = np.random.default_rng(3)
    intr = (320.0, 320.0, 320.0, 240.0)
    kinds = [(96, 10), (48, 7), (96, 10), (48, 7)]
    srv = ba.Solver()
    srv.serve_start(32, 3072, 66000, 2, max_batch=16, max_in_flight=2)
    solo = ba.Solver()
    graphs = S.make_serving_mix(2, base_seed=11)
    refs = []
    try:
        sids = []
        for m, f in kinds:
            prm = ba.WindowParams(22, m, 13, f, 2, *intr)
            sids.append(srv.session_open_window(prm))
            refs.append(ba.Window(22, m, 13, f, intr))
        gids = [srv.session_open(sc) for sc in graphs]
        for frame in range(24):
            reqs = []
            for sid, (m, f) in zip(sids, kinds):
                xy = rng.uniform([16, 16], [624, 464], (m, 2)).astype(np.float32)
                E = srv.session_frame_edges(sid, m)
                delta = rng.normal(scale=np.sqrt(0.5), size=(E, 2)).astype(np.float32)
                weight = rng.uniform(0.0, 1.0, size=(E, 2)).astype(np.float32)
                reqs.append((xy, delta, weight))
            tickets = [srv.submit_frame(sid, *r) for sid, r in zip(sids, reqs)]
            fresh = [S.refresh_factors(sc, 1000 * frame + b) for b, sc in enumerate(graphs)]
            gts = [srv.submit(gid, r.target, r.weight) for gid, r in zip(gids, fresh)]
            for tk in tickets + gts:
                st, lat = srv.wait(tk, 20000)
                assert st == 0 and lat > 0
            for b, (sid, (xy, delta, weight)) in enumerate(zip(sids, reqs)):
                w = refs[b]
                w.append(torch.tensor(xy, device="cuda"))
                p = w.problem()
                p.target.add_(torch.tensor(delta, device="cuda"))
                p.weight.copy_(torch.tensor(weight, device="cuda"))
                p0, q0 = p.poses.clone(), p.patches.clone()     # the appended state, before the solve
                solo.solve([p])
                torch.cuda.synchronize()
                assert int(p.status.item()) == 0
                d = srv.session_dims(sid)
                assert (d.n_frames, d.n_patches, d.n_edges) == tuple(p.poses.shape[:1]) + (p.patches.shape[0],
                                                                                           p.kk.shape[0])
                poses, patches = srv.session_read(sid, d.n_frames, d.n_patches)
                t0 = d.t0
                ref_p, ref_q = p.poses.cpu().numpy(), p.patches.cpu().numpy()
                p0n, q0n = p0.cpu().numpy(), q0.cpu().numpy()
                if d.n_frames > t0:
                    assert err(poses[t0:] - p0n[t0:], ref_p[t0:] - p0n[t0:]) < TOL_POSE, (frame, b)
                assert err(patches[:, 2] - q0n[:, 2], ref_q[:, 2] - q0n[:, 2]) < TOL_DEPTH, (frame, b)
                # the next frame starts the reference from the served state
                p.poses.copy_(torch.tensor(poses, device="cuda"))
                p.patches.copy_(torch.tensor(patches, device="cuda"))
        for sid in sids + gids:
            srv.session_close(sid)
    finally:
        srv.serve_stop()
        srv.close()
        solo.close()
        for w in refs:
            w.close()
