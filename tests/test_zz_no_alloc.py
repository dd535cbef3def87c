"""qt_energy_noalloc: energies without any device allocation during the call.

Some callers of this library may not call cudaMalloc while they run: code
inside a custom device allocator or memory pool (an allocation there would
re-enter it), or a host process that reserves its whole device-memory budget
at start-up and forbids allocations afterwards. qt_energy_noalloc serves them:
it runs the persistent kernel with every piece of device memory it needs inside
one static array that the library carries (QT_NOALLOC_SCRATCH_BYTES, 64 MiB),
on a plan that itself holds no device memory (opts.host_only).

These tests call it through the C ABI and check it against qt_energy on the
same graphs and angles, with the tolerances of the other GPU parity tests
(1e-10 complex128, 1e-5 complex64; per edge the larger of the relative error
of (1 - e)/2 and the absolute error of e). Each test makes calls in a row, so a
call that read what the previous call left in the shared array would show.

The file name sorts last so that pytest collects it after every other test.
"""
import numpy as np
import pytest

from paper_2204_06045_gb300 import qtgb, synth

TOL = {"c128": 1e-10, "c64": 1e-5}


def scaled_err(x, ref):
    x, ref = np.asarray(x, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    d = np.abs(x - ref)
    return float(max(np.max(d / np.abs(1.0 - ref)), np.max(d)))


def _gpu_setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_06045_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def test_plan_over_the_scratch_limit_is_rejected():
    """The size check runs before any CUDA call, so this needs no GPU: the
    N=30 p=4 networks need gigabytes of intermediates, far over 64 MiB."""
    from paper_2204_06045_gb300 import build
    build.build()
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    with qtgb.plan(n, edges, p, host_only=True) as pl:
        with pytest.raises(qtgb.QTError) as ei:
            pl.energy_noalloc(g, b)
    assert ei.value.code == qtgb.QT_ENOMEM
    assert "static scratch" in str(ei.value)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_matches_qt_energy_on_two_calls(dtype):
    _gpu_setup()
    n, p = 16, 3
    edges = synth.random_regular_graph(n, 23)
    angle_sets = [synth.angles(p, 23), synth.angles(p, 24)]
    with qtgb.plan(n, edges, p, dtype=dtype) as ref_plan, qtgb.plan(n, edges, p, dtype=dtype,
                                                                    host_only=True) as pl:
        outs = []
        for g, b in angle_sets:
            zz_ref, e_ref = ref_plan.energy(g, b)
            energies, zz = pl.energy_noalloc(g, b)
            assert scaled_err(zz, zz_ref) <= TOL[dtype]
            assert abs(energies[0] - e_ref) <= TOL[dtype] * abs(e_ref)
            outs.append(zz)
    # the two angle sets give different values: a stale result would not pass
    assert np.max(np.abs(outs[0] - outs[1])) > 1e-3


@pytest.mark.gpu
def test_noalloc_alternating_plans_and_batch():
    """Different plans share the array: A, B, A, then a batch plan."""
    _gpu_setup()
    cases = [(12, synth.ring_graph(12), 3, "c64"), (18, synth.random_regular_graph(18, 5), 2, "c128")]
    for n, edges, p, dtype in cases + cases[:1]:
        g, b = synth.angles(p, n)
        with qtgb.plan(n, edges, p, dtype=dtype) as ref_plan, qtgb.plan(n, edges, p, dtype=dtype,
                                                                        host_only=True) as pl:
            zz_ref, e_ref = ref_plan.energy(g, b)
            energies, zz = pl.energy_noalloc(g, b)
        assert scaled_err(zz, zz_ref) <= TOL[dtype]
        assert abs(energies[0] - e_ref) <= TOL[dtype] * abs(e_ref)
    graphs = synth.batch(4, 2, lo=10, hi=24, base_seed=77)
    G = np.array([gg for _, _, gg, _ in graphs])
    B = np.array([bb for _, _, _, bb in graphs])
    spec = [(n, e) for n, e, _, _ in graphs]
    with qtgb.plan_batch(spec, 2, dtype="c64") as ref_plan, qtgb.plan_batch(spec, 2, dtype="c64",
                                                                           host_only=True) as pl:
        e_ref, zz_ref = ref_plan.energy_batch(G, B)
        for _ in range(2):
            energies, zz = pl.energy_noalloc(G, B)
            assert scaled_err(zz, zz_ref) <= TOL["c64"]
            assert np.all(np.abs(energies - e_ref) <= TOL["c64"] * np.abs(e_ref))


@pytest.mark.gpu
def test_noalloc_device_buffers_on_a_stream():
    torch = _gpu_setup()
    n, p = 14, 3
    edges = synth.random_regular_graph(n, 22)
    g, b = synth.angles(p, 22)
    with qtgb.plan(n, edges, p, dtype="c64") as ref_plan, qtgb.plan(n, edges, p, dtype="c64",
                                                                    host_only=True) as pl:
        zz_ref, e_ref = ref_plan.energy(g, b)
        gd = torch.tensor(g, dtype=torch.float64, device="cuda")
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        for _ in range(2):
            en = torch.zeros(1, dtype=torch.float64, device="cuda")
            zz = torch.zeros(edges.shape[0], dtype=torch.float64, device="cuda")
            pl.energy_noalloc(gd, bd, energies=en, edge_zz=zz, stream=s)
            assert scaled_err(zz.cpu().numpy(), zz_ref) <= TOL["c64"]
            assert abs(float(en.cpu()[0]) - e_ref) <= TOL["c64"] * abs(e_ref)


@pytest.mark.gpu
def test_noalloc_batch_with_fused_units():
    """A batch whose small buckets form fused units (their programs also live
    in the static array) against qt_energy_batch, two calls in a row."""
    _gpu_setup()
    graphs = synth.batch(8, 2, lo=40, hi=120, base_seed=3000)
    spec = [(n, e) for n, e, _, _ in graphs]
    G = np.array([gg for _, _, gg, _ in graphs])
    B = np.array([bb for _, _, _, bb in graphs])
    with qtgb.plan_batch(spec, 2, dtype="c64") as ref_plan, qtgb.plan_batch(spec, 2, dtype="c64",
                                                                           host_only=True) as pl:
        assert pl.stats()["n_units"] > 0
        e_ref, zz_ref = ref_plan.energy_batch(G, B)
        for _ in range(2):
            energies, zz = pl.energy_noalloc(G, B)
            assert scaled_err(zz, zz_ref) <= TOL["c64"]
            assert np.all(np.abs(energies - e_ref) <= TOL["c64"] * np.abs(e_ref))
