"""The dispatch order of the job compiler's tables (host only, no GPU): every
series is written once; a job reads only series written in earlier layers (no
read-after-write inside a layer, the property that lets the jobs of one layer
run in any order, Sec. 5); the order is by layer and follows the dependencies;
within a layer, the jobs whose output another job reads come before the leaves
(products only the addition stage reads).  Checked on the paper's p1, a slice
of the p2-like polynomial, random polynomials with powers, their complex form
and a system."""
import numpy as np
import pytest

from paper_2101_10881_gb300 import pes, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    pes.build()


def check_schedule(jobs):
    jobs = np.asarray(jobs)
    assert jobs.ndim == 2 and jobs.shape[1] >= 4
    producer = {}
    for i, (_, _, out, layer) in enumerate(jobs[:, :4].tolist()):
        assert out not in producer, "a series is written twice"
        producer[out] = (i, layer)
    read = set(jobs[:, 0].tolist()) | set(jobs[:, 1].tolist())
    last_layer = -1
    seen_leaf_in_layer = False
    for i, (in1, in2, out, layer) in enumerate(jobs[:, :4].tolist()):
        assert layer >= last_layer, "layers out of order"
        if layer != last_layer:
            seen_leaf_in_layer = False
        last_layer = layer
        for s in (in1, in2):
            if s in producer:
                p, pl = producer[s]
                assert p < i, "a job before its producer"
                assert pl < layer, "read-after-write inside a layer"
        leaf = out not in read
        if leaf:
            seen_leaf_in_layer = True
        else:
            assert not seen_leaf_in_layer, "a chain job after a leaf of its layer"


def test_p1_schedule():
    check_schedule(pes.jobc_program(synth.supports_p1(), 16)["jobs"])


def test_p2_slice_schedule():
    check_schedule(pes.jobc_program(synth.supports_p2()[:12], 128)["jobs"])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_powers_and_complex_schedules(seed):
    rng = np.random.default_rng(seed)
    supp = synth.random_supports(rng, 9, 14, 1, 7)
    exps = [[int(e) for e in rng.integers(1, 4, size=len(s))] for s in supp]
    check_schedule(pes.jobc_program(supp, 9)["jobs"])
    check_schedule(pes.jobc_program(supp, 9, exponents=exps)["jobs"])
    check_schedule(pes.jobc_program(supp, 9, exponents=exps, complex_series=True)["jobs"])


def test_system_schedule():
    rng = np.random.default_rng(7)
    polys = [synth.random_supports(rng, 10, int(m), 2, 6) for m in (5, 0, 8, 3)]
    flat = [s for p in polys for s in p]
    check_schedule(pes.jobc_program(flat, 10, polys=[len(p) for p in polys])["jobs"])
