"""Persistent passes (MPM_OPT_PERSISTENT): every checkpoint segment of the
forward pass, the recomputation and the adjoint runs as one cooperative launch
whose CTAs walk the substeps with grid-wide barriers.  Same results as the
FP64 oracle (and so as the chained launches), in 2D and in 3D with node-block
lists, replayed as CUDA graphs or launched directly, twice in a row; and a
barrier wait that runs out of polls ends the call with MPM_ERR_TIMEOUT while
the handle stays usable."""
import functools

import numpy as np
import pytest

from paper_2503_22767_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22767_gb300 import binding as B  # noqa: E402
from paper_2503_22767_gb300.sim import Simulator  # noqa: E402
from test_gpu_parity import assert_grads, assert_state, run_gpu  # noqa: E402

CASES = {
    "walker2d_s0.5_300": lambda: W.walker_2d(seed=2, n_steps=300, scale=0.5, checkpoint_every=100),
    "batch2d_5_120": lambda: W.walker_batch_2d(seed=7, n_instances=5, n_steps=120, n_lo=1500, n_hi=6000),
    "walker3d_48_60": lambda: W.walker_3d(seed=4, n_steps=60, res=48, scale=0.25, checkpoint_every=25),
    "plate3d_32_3tasks_60": lambda: W.plate_3d(seed=3, n_steps=60, res=32, cells=(20, 5, 20)),
}


@functools.lru_cache(maxsize=None)
def _oracle(key):
    import oracle

    w = CASES[key]()
    with oracle.threads():
        return w, oracle.forward(w), oracle.backward(w, ckpt_every=25)


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("key", list(CASES))
def test_persistent_passes_match_oracle(key, graphs):
    w, of, ob = _oracle(key)
    opts = {B.MPM_OPT_PERSISTENT: 1, B.MPM_OPT_GRAPHS: graphs}
    for _ in range(2):
        g = run_gpu(w, options=opts)
        assert_state(g, of, w)
        assert_grads(g, ob, w)
        np.testing.assert_allclose(g["loss"], of["loss"], rtol=1e-3, atol=1e-7 * np.abs(of["loss"]).max())


def test_persistent_barrier_timeout_is_a_status():
    """A one-poll spin limit: the tens of CTAs of the launch do not all reach
    a barrier within one poll of each other, so a wait runs out, the kernel
    returns and the call reports MPM_ERR_TIMEOUT.  With the limit restored the
    same handle computes the oracle's results."""
    key = "walker2d_s0.5_300"
    w, of, ob = _oracle(key)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    sim = Simulator(w.cfg, options={B.MPM_OPT_PERSISTENT: 1})
    default = sim.options()
    sim.set_option(B.MPM_OPT_SPIN_LIMIT, 1)
    statuses = []
    for _ in range(3):
        try:
            sim.forward(t(w.x0), t(w.phi), t(w.mag), t(w.field), target=t(w.target), v0=t(w.v0))
            statuses.append(B.MPM_OK)
        except B.MpmError as e:
            statuses.append(e.status)
    assert B.MPM_ERR_TIMEOUT in statuses, statuses
    assert all(s in (B.MPM_OK, B.MPM_ERR_TIMEOUT) for s in statuses), statuses
    sim.set_option(B.MPM_OPT_SPIN_LIMIT, 1 << 22)
    loss, x = sim.forward(t(w.x0), t(w.phi), t(w.mag), t(w.field), target=t(w.target), v0=t(w.v0), want_x=True)
    gp, gm, gf = sim.backward(torch.ones(w.cfg.n_instances, device="cuda"))
    u, v, C, E = sim.read_state_strain()
    xs, _, _, F = sim.read_state()
    g = dict(loss=loss.cpu().numpy().astype(np.float64), x=x.cpu().numpy(), x_state=xs.cpu().numpy(),
             v=v.cpu().numpy(), C=C.cpu().numpy(), F=F.cpu().numpy(), u=u.cpu().numpy(), E=E.cpu().numpy(),
             g_phi=gp.cpu().numpy(), g_mag=gm.cpu().numpy(), g_field=gf.cpu().numpy())
    assert sim.options()["persistent"] == default["persistent"] == 1
    sim.close()
    assert_state(g, of, w)
    assert_grads(g, ob, w)
