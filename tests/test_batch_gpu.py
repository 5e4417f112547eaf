"""Batched hierarchies advanced by one persistent cooperative launch: every member
matches the same hierarchy advanced alone with the batch's interface mapping (one
node per thread; bitwise: the same device arithmetic per node) and the FP64 oracle;
the grid barrier's bounded wait reports a timeout instead of hanging."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2004_14887_gb300 import lbm  # noqa: E402
from paper_2004_14887_gb300 import workloads as W  # noqa: E402


def _small_batch(storage, n=4, seed=3):
    return W.batch2d(n=n, seed=seed, storage=storage, sides=(48, 64, 96, 128))


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_batch_members_equal_individual_runs(storage):
    descs = _small_batch(storage)
    b = lbm.Batch(descs)
    singles = []
    for d, m in zip(descs, b.members):
        s = lbm.Hierarchy(d)
        s.set_interface_mapping(lbm.IFACE_NODE)
        for l in range(m.n_levels):
            r, u = W.init_fields(d, l)
            m.init_fields(l, r, u)
            s.init_fields(l, r, u)
        singles.append(s)
    steps = 13
    b.advance(5)
    b.advance(steps - 5)
    b.check_status()
    for s in singles:
        s.advance(steps)
    for m, s in zip(b.members, singles):
        for l in range(m.n_levels):
            assert np.array_equal(m.get_pops(l), s.get_pops(l))


def test_batch_member_matches_oracle_f64():
    descs = _small_batch("f64", n=3, seed=5)
    b = lbm.Batch(descs)
    orcs = []
    for d, m in zip(descs, b.members):
        o = O.Hierarchy(d)
        for l in range(m.n_levels):
            r, u = W.init_fields(d, l)
            m.init_fields(l, r, u)
            o.init(l, r, u)
        orcs.append(o)
    b.advance(20)
    b.check_status()
    for m, o in zip(b.members, orcs):
        o.advance(20)
        for l in range(m.n_levels):
            mask = m.node_class(l) != lbm.HOLE
            rg, ug = m.get_macros(l)
            ro, uo = o.macros(l)
            assert np.max(np.abs(rg[mask] - ro[mask])) / np.max(np.abs(ro[mask])) < 1e-12
            assert np.max(np.abs(ug[:, mask] - uo[:, mask])) / np.max(np.abs(uo[:, mask])) < 1e-12


def test_batch_barrier_wait_is_bounded():
    """A block that leaves without arriving makes the others' waits run out (200 ms):
    the call returns LBM_ERR_TIMEOUT and the context stays usable."""
    descs = _small_batch("f32", n=2)
    b = lbm.Batch(descs)
    assert b.check_barrier(-1, 200000) == lbm.LBM_OK
    assert b.check_barrier(3, 200000) == lbm.LBM_ERR_TIMEOUT
    for d, m in zip(descs, b.members):
        for l in range(m.n_levels):
            r, u = W.init_fields(d, l)
            m.init_fields(l, r, u)
    b.advance(4)
    b.check_status()
    with pytest.raises(lbm.LbmError):
        b.members[0].advance(1)  # a member advances only with its batch


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_phase_launches_equal_the_persistent_launch(storage):
    """The two launch structures of a batch (one cooperative launch per coarse step, or
    one launch per phase) run the same phase bodies in the same order: bitwise equal
    members after the same steps, also when the structure changes between calls."""
    descs = _small_batch(storage)
    out = []
    for paths in ([lbm.BATCH_PERSISTENT], [lbm.BATCH_PHASES], [lbm.BATCH_PHASES, lbm.BATCH_PERSISTENT]):
        b = lbm.Batch(descs)
        for d, m in zip(descs, b.members):
            for l in range(m.n_levels):
                r, u = W.init_fields(d, l)
                m.init_fields(l, r, u)
        for p in paths:
            b.set_path(p)
            assert b.path() == p
            b.advance(6)
        b.check_status()
        out.append([[m.get_pops(l) for l in range(m.n_levels)] for m in b.members])
        b.close()
    steps = {0: 6, 1: 6, 2: 12}
    assert steps[0] == steps[1]
    for ma, mb in zip(out[0], out[1]):
        for a, c in zip(ma, mb):
            assert np.array_equal(a, c)


def test_batch_autotune_chooses_a_launch_structure():
    descs = _small_batch("f32")
    b = lbm.Batch(descs)
    for d, m in zip(descs, b.members):
        for l in range(m.n_levels):
            r, u = W.init_fields(d, l)
            m.init_fields(l, r, u)
    res = b.autotune(reps=3)
    assert res["path"] in (lbm.BATCH_PERSISTENT, lbm.BATCH_PHASES)
    assert all(t > 0 for t in res["us"])
    assert res["path"] == (lbm.BATCH_PHASES if res["us"][1] < res["us"][0] else lbm.BATCH_PERSISTENT)
    b.advance(2)
    b.check_status()
