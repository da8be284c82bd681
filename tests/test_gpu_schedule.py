"""GPU: the tensor-core schedule network against its FP64 oracle, and the learned,
audited detection schedule against the plain one."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2311_04648_gb300 import dem, workloads as W

pytestmark = pytest.mark.gpu


def test_tensor_core_forward_matches_oracle():
    rng = np.random.default_rng(3)
    p = rng.normal(scale=0.3, size=omlp.NPARAM).astype(np.float32)
    for rows in (1, 17, 333):
        X = rng.normal(size=(rows, 16)).astype(np.float32)
        got = dem.mlp_forward(p, X)
        want = omlp.forward(p.astype(np.float64), X.astype(np.float64), bf=True)
        assert np.max(np.abs(got - want)) <= 1e-3 * (1.0 + np.max(np.abs(want)))


@pytest.mark.parametrize("rows", [1, 5, 257, 1000])
def test_tensor_core_gradient_matches_oracle(rows):
    """Every parameter block (W1, b1, W2, b2, W3, b3) element by element against the
    oracle with BF16-rounded operands, within one BF16 ulp of each element (plus 2^-14
    of the block's largest entry where a sum cancels); the whole vector also in norm
    against the exact (unrounded) gradient."""
    rng = np.random.default_rng(4 + rows)
    p = rng.normal(scale=0.3, size=omlp.NPARAM).astype(np.float32)
    X = rng.normal(size=(rows, 16)).astype(np.float32)
    Y = rng.normal(size=(rows, 2)).astype(np.float32)
    L, g = dem.mlp_loss_grad(p, X, Y)
    Lo, go = omlp.loss_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), bf=True)
    assert L == pytest.approx(Lo, rel=1e-3)
    tol = omlp.gradient_tolerance(go)
    for name, sl in omlp.blocks():
        err = np.abs(g[sl].astype(np.float64) - go[sl])
        k = int(np.argmax(err - tol[sl]))
        assert np.all(err <= tol[sl]), (name, k, float(g[sl][k]), float(go[sl][k]), float(tol[sl][k]))
    # and the exact (unrounded) gradient is within BF16 accuracy
    Le, ge = omlp.loss_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), bf=False)
    assert np.linalg.norm(g - ge) <= 5e-2 * np.linalg.norm(ge)


def _scene():
    return W.settle_box(n=1500, box=(0.03, 0.03, 0.06), seed=21, vel_sigma=0.4, h=1e-6)


def test_learned_schedule_trains_and_stays_bit_identical():
    scene = _scene()
    beta = 5e-5
    teacher = dem.World.from_scene(scene, precision="voxel_fp32", schedule="velocity_bound", margin=beta,
                                   margin_max=beta)
    teacher.schedule_collect(True)
    teacher.step(1600)
    teacher.schedule_collect(False)
    st = teacher.stats()
    assert st["schedule_samples"] > 30
    loss0 = teacher.schedule_train(epochs=1, lr=1e-3, seed=1)
    loss = teacher.schedule_train(epochs=60, lr=3e-3, seed=1)
    assert loss < loss0
    blob = teacher.schedule_export()
    # a fresh world with the learned schedule and the plain every-step world
    a = dem.World.from_scene(scene, precision="voxel_fp32", schedule="every_step", margin_max=beta)
    b = dem.World.from_scene(scene, precision="voxel_fp32", schedule="learned", margin=beta, margin_max=beta)
    c = dem.World.from_scene(scene, precision="voxel_fp32", schedule="velocity_bound", margin=beta, margin_max=beta)
    b.load_schedule_model(blob)
    for w in (a, b, c):
        w.step(800)
    for xa, xb in zip(a.owner_state(), b.owner_state()):
        assert np.array_equal(xa, xb)
    for xa, xc in zip(a.owner_state(), c.owner_state()):
        assert np.array_equal(xa, xc)
    sb, sc = b.stats(), c.stats()
    cost_b = sb["rebuilds"] + 2 * sb["audit_fallbacks"]
    cost_c = sc["rebuilds"] + 2 * sc["audit_fallbacks"]
    print("learned", sb["rebuilds"], sb["audit_fallbacks"], "velocity bound", sc["rebuilds"], sc["audit_fallbacks"])
    assert cost_b < cost_c


def test_learned_schedule_gains_out_of_sample_on_a_discharging_hopper():
    """The network trained only on the method's own trajectories of other flows (the
    2,000-sphere box with random velocities and a 200,000-sphere section of the settling
    column) and then run on a 50,000-sphere conical hopper it never saw: fewer list
    rebuilds plus twice the audit fallbacks (each an inline rebuild) than the velocity
    bound, with the same trajectory bits (every step is audited)."""
    blob = None
    for sc, steps in ((W.settle_box(n=2000, vel_sigma=0.3, seed=2), 2048), (W.settling_column(n=200_000), 1536)):
        tw = dem.World.from_scene(sc, precision="voxel_fp32", schedule="velocity_bound")
        if blob is not None:
            tw.load_schedule_model(blob)
        tw.schedule_collect(True)
        tw.step(steps)
        tw.schedule_collect(False)
        tw.schedule_train(epochs=60, lr=3e-3, seed=1)
        blob = tw.schedule_export()
        tw.close()
    hopper = W.cone_hopper(n=50_000)
    runs = {}
    for sched in ("velocity_bound", "learned"):
        w = dem.World.from_scene(hopper, precision="voxel_fp32", schedule=sched, margin=6e-5, margin_max=6e-5)
        if sched == "learned":
            w.load_schedule_model(blob)
        w.step(8000)
        st = w.stats()
        runs[sched] = (st["rebuilds"] + 2 * st["audit_fallbacks"], st["rebuilds"], st["audit_fallbacks"],
                       w.owner_state())
        w.close()
    print("hopper 50k, 8000 steps: learned cost", runs["learned"][:3], "velocity bound", runs["velocity_bound"][:3])
    for a, b in zip(runs["learned"][3], runs["velocity_bound"][3]):
        assert np.array_equal(a, b)
    assert runs["learned"][0] < runs["velocity_bound"][0]
