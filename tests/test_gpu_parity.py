"""CUDA path vs the FP64 oracle, through the C ABI, on seeded synthetic scenes.

Sec. 3.1 Eq. 6: two Gauss-Newton iterations with the Schur complement; the
oracle solves the dense normal equations instead.  Every test compares element
by element (relative 2-norm per problem) on identical float32 inputs.
"""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from oracle import dense_gn as dg
from oracle import schur
from tests.gpu_util import (TOL_DEPTH, TOL_POSE, align_quats, end_to_end_errors, iteration_abs_errors,
                            iteration_errors, err, rel, scene_at, solve_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[False, True], ids=["fp32-schur", "tf32-schur"])
def solver(request):
    """Both accumulation modes of the Schur complement: compensated FP32 on the
    CUDA cores (the default) and three TF32 products on the tensor cores (opt-in)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    s = ba.Solver(schur_tf32=request.param)
    yield s
    s.close()


def step_errors(solver, scene, index, n_iters):
    """Per-iteration errors against the oracle's teacher-forced step.  In the
    default FP32 mode each increment is measured relative to itself.  The opt-in
    TF32 mode does not hold that on every scene: the tensor cores truncate their
    FP32 accumulation, and on some 8-frame scenes the relative error of the
    second (small) increment reaches ~1e-4; it is measured against the first
    increment's norm instead (the solve's own update scale), a limit of that
    mode stated with its configuration flag."""
    if solver.schur_tf32:
        return iteration_abs_errors(solver, scene, index, n_iters)
    return iteration_errors(solver, scene, index, n_iters)


def test_reduced_system_matches_oracle_schur(solver):
    for spec, seed in [(S.PLAIN_N8, 0), (S.WINDOW_N22, 1)]:
        sc = S.make_scene(spec, seed)
        prob = ba.problem_from_scene(sc)
        Sg, vg = solver.reduced_system(prob)
        torch.cuda.synchronize()
        pr = dg.Problem.from_scene(sc)
        Sr, vr = schur.reduced_system(pr, pr.T, pr.d)
        assert err(Sg.cpu().numpy(), Sr) < 2e-6
        assert err(vg.cpu().numpy(), vr) < 2e-6


@pytest.mark.parametrize("spec,seed", [(S.PLAIN_N8, 3), (S.PLAIN_N8, 4), (S.WINDOW_N22, 5)])
def test_each_iteration_matches_oracle_step(solver, spec, seed):
    sc = S.make_scene(spec, seed)
    probs = solve_gpu(solver, [sc])
    assert int(probs[0].status.item()) == 0
    for t, (e_xi, e_dd) in enumerate(step_errors(solver, sc, 0, sc.n_iters)):
        assert e_xi < TOL_POSE, (t, e_xi)
        assert e_dd < TOL_DEPTH, (t, e_dd)


@pytest.mark.parametrize("spec,seed", [(S.PLAIN_N8, 6), (S.WINDOW_N22, 7)])
def test_whole_solve_matches_oracle(solver, spec, seed):
    sc = S.make_scene(spec, seed)
    probs = solve_gpu(solver, [sc])
    e_pose, e_depth, ref = end_to_end_errors(sc, probs[0])
    assert e_pose < TOL_POSE and e_depth < TOL_DEPTH, (e_pose, e_depth)
    # free-running second increment (the iterates differ by FP32 rounding)
    _, _, dxi2 = solver.iterate(0, 1, sc.n_frames, sc.n_patches, sc.t0)
    assert err(dxi2, ref["dxi"][1]) < 1e-3


@pytest.mark.parametrize("spec,seed,min_off", [(dataclasses.replace(S.PLAIN_N8, near_frac=0.5), 6, 8),
                                                (dataclasses.replace(S.PLAIN_N8, near_frac=0.3), 2, 3),
                                                (dataclasses.replace(S.WINDOW_N22, near_frac=0.1), 1, 200)])
def test_edges_behind_the_camera_match_oracle(solver, spec, seed, min_off):
    """Scenes with patches close to their source camera, seen from behind by
    cameras further along the path: those edges' homogeneous depth is far below
    z_min (0.1 or more from the threshold at every oracle iterate), so both
    paths must leave them out.  Per-iteration and whole-solve parity.  The
    seeds are ones whose reduced system is no more sensitive than the regular
    scenes' (a 1e-7 relative perturbation of the Schur sum moves the pose
    increment by < 5e-6, measured with the oracle): on some 8-frame near-patch
    scenes it moves it by ~1e-4, beyond what any FP32 Schur sum can meet."""
    sc = S.make_scene(spec, seed)
    pr = dg.Problem.from_scene(sc)
    T, d = pr.T.copy(), pr.d.copy()
    for _ in range(sc.n_iters + 1):
        Z = dg.reproject(pr, T, d)[1][:, 2]
        assert (Z <= dg.Z_MIN).sum() >= min_off
        assert np.abs(Z - dg.Z_MIN).min() > 0.1
        T, d, _, _ = dg.gn_step(pr, T, d)
    probs = solve_gpu(solver, [sc])
    assert int(probs[0].status.item()) == 0
    for t, (e_xi, e_dd) in enumerate(step_errors(solver, sc, 0, sc.n_iters)):
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH, (t, e_xi, e_dd)
    e_pose, e_depth, _ = end_to_end_errors(sc, probs[0])
    assert e_pose < TOL_POSE and e_depth < TOL_DEPTH, (e_pose, e_depth)


def test_batched_mix_matches_solving_alone(solver):
    """Problems of different shapes in one batch give the same results as
    each problem solved by itself (the reduction order differs, so within
    tolerance rather than bitwise)."""
    specs = [S.PLAIN_N8, S.WINDOW_N22, dataclasses.replace(S.WINDOW_N22, patches_per_frame=48, radius=8),
             dataclasses.replace(S.PLAIN_N8, n_frames=12, t0=4, radius=5)]
    scenes = [S.make_scene(sp, 20 + i) for i, sp in enumerate(specs)]
    alone = [solve_gpu(solver, [sc])[0] for sc in scenes]
    mixed = solve_gpu(solver, scenes)
    for a, m, sc in zip(alone, mixed, scenes):
        assert int(m.status.item()) == 0
        pa, pm = a.poses.cpu().numpy(), m.poses.cpu().numpy()
        assert err(pm[sc.t0:] - sc.poses[sc.t0:], pa[sc.t0:] - sc.poses[sc.t0:]) < 1e-5
        da, dm = a.patches[:, 2].cpu().numpy(), m.patches[:, 2].cpu().numpy()
        assert err(dm - sc.patches[:, 2], da - sc.patches[:, 2]) < 1e-5
    for i in range(len(scenes)):
        for t, (e_xi, e_dd) in enumerate(step_errors(solver, scenes[i], i, scenes[i].n_iters)):
            assert e_xi < TOL_POSE and e_dd < TOL_DEPTH, (i, t, e_xi, e_dd)


def test_repeated_solves_are_bitwise_identical(solver):
    sc = S.make_scene(S.WINDOW_N22, 30)
    a = solve_gpu(solver, [sc])[0]
    b = solve_gpu(solver, [sc])[0]
    assert torch.equal(a.poses, b.poses) and torch.equal(a.patches, b.patches)


# ---------------------------------------------------------------- edge cases

def _drop_edges(sc, frac, seed):
    rng = np.random.default_rng(seed)
    keep = rng.uniform(size=sc.n_edges) >= frac
    return dataclasses.replace(sc, kk=sc.kk[keep], jj=sc.jj[keep], target=sc.target[keep],
                               weight=sc.weight[keep], outlier=sc.outlier[keep], uv_true=sc.uv_true[keep])


def test_ragged_graph_with_missing_edges_and_isolated_patches(solver):
    sc = S.make_scene(dataclasses.replace(S.WINDOW_N22, patches_per_frame=37), 40)
    sc = _drop_edges(sc, 0.3, 1)
    # patch 5 loses every edge: its inverse depth must not move
    keep = sc.kk != 5
    sc = dataclasses.replace(sc, kk=sc.kk[keep], jj=sc.jj[keep], target=sc.target[keep], weight=sc.weight[keep],
                             outlier=sc.outlier[keep], uv_true=sc.uv_true[keep])
    probs = solve_gpu(solver, [sc])
    assert int(probs[0].status.item()) == 0
    for e_xi, e_dd in step_errors(solver, sc, 0, sc.n_iters):
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH
    assert probs[0].patches[5, 2].item() == sc.patches[5, 2]


def test_no_self_edges_and_uneven_frames(solver):
    sc = S.make_scene(dataclasses.replace(S.PLAIN_N8, patches_per_frame=70, n_frames=9, t0=3), 41)
    keep = sc.anchor[sc.kk] != sc.jj
    sc = dataclasses.replace(sc, kk=sc.kk[keep], jj=sc.jj[keep], target=sc.target[keep], weight=sc.weight[keep],
                             outlier=sc.outlier[keep], uv_true=sc.uv_true[keep])
    solve_gpu(solver, [sc])
    for e_xi, e_dd in step_errors(solver, sc, 0, 2):
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH


def test_all_poses_fixed_updates_depths_only(solver):
    sc = S.make_scene(dataclasses.replace(S.PLAIN_N8, t0=8), 42)
    probs = solve_gpu(solver, [sc])
    assert torch.equal(probs[0].poses.cpu(), torch.as_tensor(sc.poses))
    ref = dg.solve_scene(sc)
    d = probs[0].patches[:, 2].cpu().numpy()
    assert err(d - sc.patches[:, 2], ref["depths"] - sc.patches[:, 2]) < TOL_DEPTH


@pytest.mark.parametrize("nf", [1, 15])
def test_extreme_free_pose_counts(solver, nf):
    spec = dataclasses.replace(S.PLAIN_N8, n_frames=17, patches_per_frame=24, radius=6, t0=17 - nf)
    sc = S.make_scene(spec, 43 + nf)
    probs = solve_gpu(solver, [sc])
    assert int(probs[0].status.item()) == 0
    for e_xi, e_dd in step_errors(solver, sc, 0, 2):
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH


def test_more_iterations(solver):
    """Five iterations: the first two match relatively; once the increments
    reach the FP32 floor they are compared against the first increment."""
    sc = S.make_scene(dataclasses.replace(S.PLAIN_N8, n_iters=5), 44)
    solve_gpu(solver, [sc])
    for e_xi, e_dd in step_errors(solver, sc, 0, 5)[:2]:
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH
    for e_xi, e_dd in iteration_abs_errors(solver, sc, 0, 5):
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH


def test_batch_with_different_iteration_counts(solver):
    """Problems with 1, 3 and 2 iterations in one batch: the one-iteration
    problem takes its last depth update inside the second linearisation
    launch, the others in the launches that follow; each result equals the
    problem solved alone within the parity tolerance (the batch splits the
    Schur sums differently, and three iterations carry the rounding
    differences further: 1.1e-5 measured on the depths) and the caller's
    status and poses are written back."""
    specs = [dataclasses.replace(S.PLAIN_N8, n_iters=1), dataclasses.replace(S.WINDOW_N22, n_iters=3),
             dataclasses.replace(S.PLAIN_N8, n_frames=12, t0=4, radius=5)]
    scenes = [S.make_scene(sp, 60 + i) for i, sp in enumerate(specs)]
    alone = [solve_gpu(solver, [sc])[0] for sc in scenes]
    mixed = solve_gpu(solver, scenes)
    for a, m, sc in zip(alone, mixed, scenes):
        assert int(m.status.item()) == 0 and int(a.status.item()) == 0
        pa, pm = a.poses.cpu().numpy(), m.poses.cpu().numpy()
        assert not np.array_equal(pm[sc.t0:], sc.poses[sc.t0:])
        assert err(pm[sc.t0:] - sc.poses[sc.t0:], pa[sc.t0:] - sc.poses[sc.t0:]) < TOL_POSE
        da, dm = a.patches[:, 2].cpu().numpy(), m.patches[:, 2].cpu().numpy()
        assert err(dm - sc.patches[:, 2], da - sc.patches[:, 2]) < TOL_DEPTH
    for i in range(len(scenes)):
        for e_xi, e_dd in step_errors(solver, scenes[i], i, scenes[i].n_iters)[:2]:
            assert e_xi < TOL_POSE and e_dd < TOL_DEPTH
        for e_xi, e_dd in iteration_abs_errors(solver, scenes[i], i, scenes[i].n_iters):
            assert e_xi < TOL_POSE and e_dd < TOL_DEPTH


def test_empty_graph_is_not_spd_and_leaves_state(solver):
    sc = S.make_scene(S.PLAIN_N8, 45)
    sc = dataclasses.replace(sc, kk=sc.kk[:0], jj=sc.jj[:0], target=sc.target[:0], weight=sc.weight[:0])
    probs = solve_gpu(solver, [sc])
    assert int(probs[0].status.item()) & ba.STATUS_NOT_SPD
    assert torch.equal(probs[0].poses.cpu(), torch.as_tensor(sc.poses))
    assert torch.equal(probs[0].patches.cpu(), torch.as_tensor(sc.patches))


@pytest.mark.parametrize("breakage", ["unsorted_kk", "frame_out_of_range", "duplicate_edge", "anchor_order",
                                      "duplicate_at_quad_start", "unsorted_at_warp_start"])
def test_bad_input_is_flagged_and_leaves_state(solver, breakage):
    """Ordering and range violations anywhere in the edge list, including at
    the first edge of a 4-edge group (its predecessor comes from the
    neighbouring thread) and at the first edge of a warp's span (read on its
    own); every patch of this scene has 8 edges, so edges 128..135 are patch 16."""
    sc = S.make_scene(S.PLAIN_N8, 46)
    kk, jj, anchor = sc.kk.copy(), sc.jj.copy(), sc.anchor.copy()
    if breakage == "unsorted_kk":
        kk[10], kk[500] = kk[500], kk[10]
    elif breakage == "frame_out_of_range":
        jj[7] = sc.n_frames
    elif breakage == "duplicate_edge":
        jj[9] = jj[8]
    elif breakage == "duplicate_at_quad_start":
        assert kk[132] == kk[131]
        jj[132] = jj[131]
    elif breakage == "unsorted_at_warp_start":
        kk[128] = kk[127] - 1
    else:
        anchor[3], anchor[400] = anchor[400], anchor[3]
    bad = dataclasses.replace(sc, kk=kk, jj=jj, anchor=anchor)
    good = S.make_scene(S.PLAIN_N8, 47)
    probs = solve_gpu(solver, [bad, good])
    assert int(probs[0].status.item()) == ba.STATUS_BAD_INPUT
    assert torch.equal(probs[0].poses.cpu(), torch.as_tensor(sc.poses))
    assert torch.equal(probs[0].patches.cpu(), torch.as_tensor(sc.patches))
    # the good problem in the same batch is unaffected
    assert int(probs[1].status.item()) == 0
    for e_xi, e_dd in step_errors(solver, good, 1, 2):
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH


@pytest.mark.parametrize("kk_off,jj_off,drop", [(1, 1, 1), (2, 2, 3), (3, 3, 2), (0, 1, 0), (3, 1, 2)])
def test_edge_arrays_at_any_offset_solve_identically(solver, kk_off, jj_off, drop):
    """kk and jj at every 4-byte offset from a 16-byte boundary, with edge
    counts that leave 0-3 edges over after the 4-edge groups: the plan reads
    the edges in groups of four where kk and jj share their offset (a short
    head and tail edge by edge) and edge by edge where they do not; every
    placement gives bitwise the same solve."""
    sc = S.make_scene(S.WINDOW_N22, 50)
    if drop:
        sc = dataclasses.replace(sc, kk=sc.kk[:-drop], jj=sc.jj[:-drop], target=sc.target[:-drop],
                                 weight=sc.weight[:-drop], outlier=sc.outlier[:-drop], uv_true=sc.uv_true[:-drop])
    ref = solve_gpu(solver, [sc])[0]
    assert int(ref.status.item()) == 0

    def shifted(t, off):
        big = torch.zeros(t.numel() + 4, dtype=t.dtype, device=t.device)
        big[off:off + t.numel()] = t
        return big[off:off + t.numel()]

    p = ba.problem_from_scene(sc)
    p = dataclasses.replace(p, kk=shifted(p.kk, kk_off), jj=shifted(p.jj, jj_off))
    assert (p.kk.data_ptr() - kk_off * 4) % 16 == 0 and (p.jj.data_ptr() - jj_off * 4) % 16 == 0
    solver.solve([p])
    torch.cuda.synchronize()
    assert int(p.status.item()) == 0
    assert torch.equal(p.poses, ref.poses) and torch.equal(p.patches, ref.patches)


def test_host_buffer_entry_point_matches_device_entry_point(solver):
    sc = S.make_scene(S.PLAIN_N8, 48)
    dev = solve_gpu(solver, [sc])[0]
    h = dict(poses=sc.poses.copy(), patches=sc.patches.copy(), anchor=sc.anchor.copy(), kk=sc.kk.copy(),
             jj=sc.jj.copy(), target=sc.target.copy(), weight=sc.weight.copy(),
             status=np.zeros(1, np.int32), intrinsics=sc.intrinsics, t0=sc.t0, n_iters=sc.n_iters)
    solver.solve_host([h])
    assert h["status"][0] == 0
    assert np.array_equal(h["poses"], dev.poses.cpu().numpy())
    assert np.array_equal(h["patches"], dev.patches.cpu().numpy())


def test_host_buffer_entry_point_in_sub_batches(solver):
    """72 problems through the host-buffer entry point go in two sub-batches of
    36 (inputs copied on the handle's copy stream, each sub-batch solved once
    its inputs landed).  Every problem's result matches the same problem solved
    from device buffers in one batch of 72, within the parity tolerance (the
    batches split the Schur sums over different numbers of CTAs), and
    afterwards the iterates of the last sub-batch are readable."""
    scenes = [S.make_scene(S.PLAIN_N8, 700 + (b % 6)) for b in range(72)]
    dev = solve_gpu(solver, scenes)
    hs = [dict(poses=sc.poses.copy(), patches=sc.patches.copy(), anchor=sc.anchor.copy(), kk=sc.kk.copy(),
               jj=sc.jj.copy(), target=sc.target.copy(), weight=sc.weight.copy(),
               status=np.zeros(1, np.int32), intrinsics=sc.intrinsics, t0=sc.t0, n_iters=sc.n_iters)
          for sc in scenes]
    solver.solve_host(hs)
    for b, (h, sc) in enumerate(zip(hs, scenes)):
        assert h["status"][0] == 0, b
        t0 = sc.t0
        dp = dev[b].poses.cpu().numpy().astype(np.float64) - sc.poses
        hp = h["poses"].astype(np.float64) - sc.poses
        assert err(hp[t0:], dp[t0:]) < TOL_POSE, b
        dd = dev[b].patches[:, 2].cpu().numpy().astype(np.float64) - sc.patches[:, 2]
        hd = h["patches"][:, 2].astype(np.float64) - sc.patches[:, 2]
        assert err(hd, dd) < TOL_DEPTH, b
    poses, _, _ = solver.iterate(0, scenes[36].n_iters, scenes[36].n_frames, scenes[36].n_patches, scenes[36].t0)
    assert np.array_equal(poses, hs[36]["poses"])


def test_invalid_arguments_return_einval(solver):
    sc = S.make_scene(S.PLAIN_N8, 49)
    p = ba.problem_from_scene(sc)
    with pytest.raises(ba.BAError) as e:
        solver.solve([dataclasses.replace(p, t0=-1)])
    assert e.value.code == ba.EINVAL
    with pytest.raises(ba.BAError):
        solver.solve([dataclasses.replace(p, t0=0, poses=torch.zeros(33, 7, device="cuda"))])   # 33 free > 32


@pytest.mark.parametrize("spec,seed", [(S.PLAIN_N8, 31), (S.WINDOW_N22, 32)])
def test_reduced_solve_f64_mode_matches_oracle_and_default(spec, seed):
    """reduced_solve_f64 = 1 takes the FP64 elimination for every reduced
    system, the path the default mode falls back to when an FP32 pivot fails
    or the refinement stalls.  Per iteration it meets the oracle's step, and
    its increments agree with the default mode's FP32 factor refined in FP64
    (both solve the same FP64 system; the refinement stops within 1e-6 of
    the solution, relative)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sc = S.make_scene(spec, seed)
    f64 = ba.Solver(reduced_solve_f64=True)
    dflt = ba.Solver()
    try:
        pf = solve_gpu(f64, [sc])
        pd = solve_gpu(dflt, [sc])
        assert int(pf[0].status.item()) == int(pd[0].status.item()) == 0
        for t, (e_xi, e_dd) in enumerate(iteration_errors(f64, sc, 0, sc.n_iters)):
            assert e_xi < TOL_POSE and e_dd < TOL_DEPTH, (t, e_xi, e_dd)
        _, _, dxi_f = f64.iterate(0, 0, sc.n_frames, sc.n_patches, sc.t0)
        _, _, dxi_d = dflt.iterate(0, 0, sc.n_frames, sc.n_patches, sc.t0)
        assert err(dxi_d, dxi_f) < 1e-5
    finally:
        f64.close()
        dflt.close()


def test_ill_conditioned_reduced_system_takes_the_fp64_elimination(solver):
    """The default reduced solve (FP32 factor, FP64 refinement) must hand a
    system it cannot refine to its FP64 elimination.  The last free pose of an
    8-frame scene keeps four observations, two at full weight and two at 1e-6
    (every other edge touching it weightless), so that some of its directions
    are pinned only by the weak pair: the reduced system is SPD with condition
    number ~1.7e10, beyond what the FP32 factor's refinement contracts (at
    weight 1e-5, condition ~1.6e9, it still converges; at 1e-8 the system is no
    longer SPD in FP64 and both modes report NOT_SPD).  Checked three ways:
    status OK; the increment is bit for bit that of reduced_solve_f64 (which
    always eliminates in FP64) on the same inputs, so the FP64 elimination
    produced it; and it solves the device's own reduced system (S, v') to
    within 1e-5 relative of numpy's dense solve of that system (measured
    ~4e-7; S's two triangles differ by ~7e-9 of its largest entry, which at
    this condition number alone allows differences of that size).  At this
    condition number the FP32 linearisation moves the solution by far more
    than 1e-4 in the weak directions, so the oracle's FP64 step is no
    yardstick here."""
    sc = S.make_scene(S.PLAIN_N8, 7)
    last = sc.n_frames - 1
    w = sc.weight.copy()
    w[(sc.jj == last) | (sc.anchor[sc.kk] == last)] = 0.0
    cand = np.flatnonzero((sc.jj == last) & (sc.anchor[sc.kk] != last))
    pick = np.random.default_rng(0).choice(cand, 4, replace=False)
    w[pick[:2]] = 1.0
    w[pick[2:]] = 1e-6
    sc = dataclasses.replace(sc, weight=w.astype(np.float32))
    S_dev, v_dev = solver.reduced_system(ba.problem_from_scene(sc))
    torch.cuda.synchronize()
    Sm, vm = S_dev.cpu().numpy(), v_dev.cpu().numpy()
    assert np.abs(Sm - Sm.T).max() <= 1e-7 * np.abs(Sm).max()
    assert np.linalg.eigvalsh(0.5 * (Sm + Sm.T)).min() > 0
    cond = np.linalg.cond(Sm)
    assert 1e9 < cond < 1e11, cond
    f64 = ba.Solver(schur_tf32=solver.schur_mode, reduced_solve_f64=True)   # the same Schur mode
    try:
        pd = solve_gpu(solver, [sc])
        pf = solve_gpu(f64, [sc])
        assert int(pd[0].status.item()) == int(pf[0].status.item()) == 0
        _, _, dxi_d = solver.iterate(0, 0, sc.n_frames, sc.n_patches, sc.t0)
        _, _, dxi_f = f64.iterate(0, 0, sc.n_frames, sc.n_patches, sc.t0)
        assert np.array_equal(dxi_d, dxi_f)
        x = np.linalg.solve(Sm, vm)
        assert np.linalg.norm(dxi_d.reshape(-1) - x) <= 1e-5 * np.linalg.norm(x), cond
    finally:
        f64.close()
