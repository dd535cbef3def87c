"""GPU parity of qt_contract_* (the paper's "tncontract" expressions, §II-E):
contractions of tensors over binary indices run by the bucket-elimination
kernel, against the oracle's complex128 contraction (oracle.contract, itself
pinned to the brute-force sum) and torch.einsum on the same device.

Tolerances: complex128 within 1e-12 of the largest output magnitude,
complex64 within 1e-5 of it (FP32 products and pair sums over at most 2^25
terms).
"""
import numpy as np
import pytest

import oracle
from paper_2204_06045_gb300 import qtgb, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = {"c64": 1e-5, "c128": 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_06045_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _tdt(dtype):
    return torch.complex64 if dtype == "c64" else torch.complex128


def run(labels, out_labels, arrays, dtype, stream=None, c=None):
    ops = [torch.as_tensor(a, dtype=_tdt(dtype), device="cuda").contiguous() for a in arrays]
    out = torch.full((2,) * len(out_labels), float("nan"), dtype=_tdt(dtype), device="cuda")
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())  # the operands' copies first
    own = c is None
    if own:
        c = qtgb.contraction(labels, out_labels, dtype=dtype)
    try:
        c.run(ops, out, stream=stream)
        if stream is not None:
            c.sync(stream)
    finally:
        if own:
            c.close()
    return out.cpu().numpy()


def close(got, ref, dtype):
    scale = max(1.0, float(np.abs(ref).max()))
    return float(np.abs(got - ref).max()) <= TOL[dtype] * scale


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("seed", range(12))
def test_random_expressions_match_oracle(dtype, seed):
    la, lb, lo = synth.tncontract_random(seed, n_lo=4, n_hi=16)
    A = synth.tensor_entries(len(la), 100 + seed)
    B = synth.tensor_entries(len(lb), 200 + seed)
    ref = oracle.contract([A, B], [la, lb], lo)
    got = run([la, lb], lo, [A, B], dtype)
    assert got.shape == ref.shape and close(got, ref, dtype), (la, lb, lo)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_paper_examples(dtype):
    """The two expressions the paper prints (§II-E): dacb,ad->bcd and caedb,eab->cde."""
    for la, lb, lo in (([3, 0, 2, 1], [0, 3], [1, 2, 3]), ([2, 0, 4, 3, 1], [4, 0, 1], [2, 3, 4])):
        A, B = synth.tensor_entries(len(la), 5), synth.tensor_entries(len(lb), 6)
        assert close(run([la, lb], lo, [A, B], dtype), oracle.contract([A, B], [la, lb], lo), dtype)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_merged_and_edge_cases(dtype):
    """Merged eliminations (two summed labels, 2^13 outputs), a scalar output,
    a rank-1 operand (folded into the gate table), three operands, an output
    in reversed label order."""
    cases = [
        ([list(range(15)), [3, 9]], [x for x in range(15) if x not in (3, 9)]),
        ([[0, 1, 2, 3, 4], [4, 2, 0]], []),
        ([[5, 1, 7, 0, 2, 6], [7]], [6, 2, 0, 1, 5]),
        ([[0, 1, 2, 3, 4, 5, 6], [1, 3], [5, 6, 0]], [0, 2, 4, 6]),
        ([list(range(12)), [11, 0]], list(range(10, 0, -1))),
    ]
    for k, (labels, lo) in enumerate(cases):
        arrays = [synth.tensor_entries(len(L), 40 + 3 * k + i) for i, L in enumerate(labels)]
        if k == 0:
            with qtgb.contraction(labels, lo, dtype=dtype, host_only=True) as h:
                assert h.stats()["n_merged"] >= 1
        assert close(run(labels, lo, arrays, dtype), oracle.contract(arrays, labels, lo), dtype), k


def test_wide_expression_matches_oracle_and_torch_einsum():
    """A 24-index expression (2^24 complex64 entries, 128 MB) of the paper's
    kind: every output against the oracle, and against torch.einsum."""
    la = list(np.random.default_rng(7).permutation(24))
    lb = [int(la[3]), int(la[17]), int(la[20])]
    lo = [int(x) for x in la if x not in (la[3], la[17])][::-1]
    la = [int(x) for x in la]
    A = synth.tensor_entries(24, 77)
    B = synth.tensor_entries(3, 78)
    ref = oracle.contract([A, B], [la, lb], lo)
    got = run([la, lb], lo, [A, B], "c64")
    assert close(got, ref, "c64")
    names = "abcdefghijklmnopqrstuvwxyz"
    spec = "".join(names[x] for x in la) + "," + "".join(names[x] for x in lb) + "->" + "".join(names[x] for x in lo)
    ta = torch.as_tensor(A, dtype=torch.complex64, device="cuda")
    tb = torch.as_tensor(B, dtype=torch.complex64, device="cuda")
    assert close(got, torch.einsum(spec, ta, tb).cpu().numpy(), "c64")


def test_two_runs_on_a_stream_and_plan_reuse():
    """A plan runs again with new operands; with a stream the call only
    enqueues, and qt_contract_sync reports the kernel-side status."""
    la, lb, lo = synth.tncontract_random(31, n_lo=12, n_hi=14)
    s = torch.cuda.Stream()
    with qtgb.contraction([la, lb], lo, dtype="c64") as c:
        for rep in range(2):
            A = synth.tensor_entries(len(la), 300 + rep)
            B = synth.tensor_entries(len(lb), 400 + rep)
            got = run([la, lb], lo, [A, B], "c64", stream=s, c=c)
            assert close(got, oracle.contract([A, B], [la, lb], lo), "c64")


def test_invalid_expressions_are_refused():
    for labels, lo in (([[0, 1], [2, 3]], [0, 1, 2, 3]),   # nothing summed
                       ([[0, 0]], [0]),                      # a repeated label
                       ([[0, 1]], [5]),                      # an output label no operand has
                       ([[0, 1], [2, 3]], [1, 3]),           # two pieces: an outer product
                       ([[0, 1, 2], [1]], [1, 2])):          # an operand of output labels only
        with pytest.raises(qtgb.QTError) as ei:
            qtgb.contraction(labels, lo)
        assert ei.value.code == qtgb.QT_EINVAL, labels
