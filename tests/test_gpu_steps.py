"""The time loop on the GPU (Section 3's BDF2 recurrence, BDF1 start): five consecutive steps
against the oracle, checkpoint / resume bit for bit, and the per-step diagnostics."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import theta_basin  # noqa: E402
from oracle import fem, step as ostep  # noqa: E402
from test_oracle_fem import small_basin  # noqa: E402
from workloads import box_basin, ocean_basin  # noqa: E402

import paper_1207_0486_gb300 as pm  # noqa: E402

pytestmark = pytest.mark.gpu

NSTEPS = 5


def _case(name):
    b = {"box16": lambda: theta_basin(box_basin()),
         "ocean48": lambda: ocean_basin(nx=48, ny=40, nz=9, dx=1e5),
         "small": lambda: theta_basin(small_basin())}[name]()
    return b, pm.assemble_operator(b)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _opts(name):
    # attainable tolerances: the thin ocean basin's pressure system floors near 1e-9 in FP64
    vtol, ptol, bar = (1e-11, 2e-9, 1e-5) if name == "ocean48" else (1e-12, 1e-12, 1e-8)
    vel = pm.Options(rtol=vtol, prec=pm.PREC_IC0, max_restarts=5)
    pres = pm.Options(rtol=ptol, prec=pm.PREC_LINE, max_restarts=5)
    oopt = ostep.StepOptions(vel_rtol=vtol, pres_rtol=ptol, pres_prec="line")
    return vel, pres, oopt, bar


def _run(op, st, t1, t2, vel, pres, steps):
    for _ in range(steps):
        pm.project_step(op, st, t1, t2, vel, pres, allow_not_converged=True)


def _fields(st):
    return [st.field(f).cpu().numpy() for f in range(pm.FIELD_Q + 1)]


@pytest.mark.parametrize("name", ["box16", "ocean48"])
def test_time_loop_matches_oracle(name):
    b, op = _case(name)
    ops = fem.assemble(b)
    vel, pres, oopt, bar = _opts(name)
    st = pm.State(op)
    ost = ostep.initial_state(ops.n)
    t1, t2 = _dev(op.column_field(b.theta[0])), _dev(op.column_field(b.theta[1]))
    for k in range(NSTEPS):
        stats = pm.project_step(op, st, t1, t2, vel, pres, allow_not_converged=True)
        rep = ostep.project_step(ops, ost, oopt)
        assert st.step_index == k + 1 == ost.step
        u1, u2, u3, p = [t.cpu().numpy() for t in st.get()]
        for nm, g, o in (("u1", u1, ost.u[0]), ("u2", u2, ost.u[1]), ("u3", u3, ost.u[2]), ("p", p, ost.p)):
            scale = np.abs(o).max()
            assert np.abs(g - o).max() <= bar * scale, (name, k, nm, np.abs(g - o).max() / scale)
        if k >= 1:   # from the first BDF2 step on, every system of the step has work to do
            assert all(s.iters > 0 for s in stats[:4]), [s.iters for s in stats[:4]]
        d = st.diagnostics()
        od = ostep.diagnostics(ops, ost, rep.u_tilde)
        assert d["kinetic_energy"] == pytest.approx(od["kinetic_energy"], rel=10 * bar, abs=0)
        assert d["div_u_tilde"] == pytest.approx(od["div_u_tilde"], rel=10 * bar, abs=0)
        # div u is what the correction leaves: compared against the prediction's size
        assert abs(d["div_u"] - od["div_u"]) <= 1e-4 * od["div_u"] + 10 * bar * od["div_u_tilde"]
        assert d["div_u"] < d["div_u_tilde"]
        assert abs(d["p_mean"] - od["p_mean"]) <= bar * np.abs(ost.p).max()


@pytest.mark.parametrize("name", ["box16", "ocean48"])
def test_checkpoint_resume_is_bit_identical(name, tmp_path):
    b, op = _case(name)
    vel, pres, _, _ = _opts(name)
    t1, t2 = _dev(op.column_field(b.theta[0])), _dev(op.column_field(b.theta[1]))
    ref = pm.State(op)
    _run(op, ref, t1, t2, vel, pres, NSTEPS)
    first = pm.State(op)
    _run(op, first, t1, t2, vel, pres, 2)
    path = str(tmp_path / "state.pmck")
    first.save(path)
    assert not os.path.exists(path + ".tmp")
    with open(path, "rb") as fh:
        head = fh.read(4096)
    assert head.endswith(b"\n") and b'"step":2' in head and b'"byte_order":"little"' in head
    assert os.path.getsize(path) == 4096 + 8 * 8 * op.n
    resumed = pm.State(op)
    resumed.load_checkpoint(path)
    assert resumed.step_index == 2
    _run(op, resumed, t1, t2, vel, pres, NSTEPS - 2)
    for f, (a, c) in enumerate(zip(_fields(ref), _fields(resumed))):
        assert np.array_equal(a, c), f
    assert ref.diagnostics() == resumed.diagnostics()
    # the in-memory snapshot continues identically too
    again = pm.State(op)
    again.restore(first.snapshot())
    _run(op, again, t1, t2, vel, pres, NSTEPS - 2)
    assert all(np.array_equal(a, c) for a, c in zip(_fields(ref), _fields(again)))


def test_checkpoint_rejects_another_basin_and_damaged_files(tmp_path):
    b, op = _case("box16")
    vel, pres, _, _ = _opts("box16")
    t1, t2 = _dev(op.column_field(b.theta[0])), _dev(op.column_field(b.theta[1]))
    st = pm.State(op)
    _run(op, st, t1, t2, vel, pres, 2)
    path = str(tmp_path / "a.pmck")
    st.save(path)
    other_b, other = _case("small")
    ost = pm.State(other)
    with pytest.raises(pm.PMError) as ei:
        ost.load_checkpoint(path)
    assert ei.value.status == pm.PM_EINVAL and "another basin" in str(ei.value)
    target = pm.State(op)
    _run(op, target, t1, t2, vel, pres, 1)
    before = _fields(target)
    raw = bytearray(open(path, "rb").read())
    damaged = str(tmp_path / "flip.pmck")
    raw2 = bytearray(raw)
    raw2[4096 + 8 * 100 + 3] ^= 0x10          # one bit of u1[100]
    open(damaged, "wb").write(bytes(raw2))
    short = str(tmp_path / "short.pmck")
    open(short, "wb").write(bytes(raw[:-8]))
    for bad, word in ((damaged, "hash"), (short, "payload size"), (str(tmp_path / "missing.pmck"), "cannot open")):
        with pytest.raises(pm.PMError) as ei:
            target.load_checkpoint(bad)
        assert ei.value.status == pm.PM_EINVAL and word in str(ei.value), (bad, str(ei.value))
        assert target.step_index == 1
        assert all(np.array_equal(a, c) for a, c in zip(before, _fields(target)))
