"""The complex64 probability and rescaling that the kernels form without
float<->double conversion instructions give the bits of the conversion
instructions, over random bit patterns, subnormals and exact ties."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_07816_b300 import sv as _sv
    _sv.load_library()
    return _sv


@pytest.mark.parametrize("which", [0, 1])
def test_integer_pipe_matches_fp64(sv, which):
    for seed in (1, 2, 3):
        bad, first = sv.sv_selftest(which, 20_000_000, seed)
        assert bad == 0, f"which={which} seed={seed}: {bad} mismatches, first case {first}"


def test_selftest_rejects_bad_arguments(sv):
    with pytest.raises(sv.SVError):
        sv.sv_selftest(3, 10)


def test_bounded_wait_reports_timeout_and_context_survives(sv):
    """A look-back wait on a descriptor nothing publishes gives up, flags a
    timeout and returns; the device then keeps working."""
    bad, flags = sv.sv_selftest(2, 0)
    assert bad == 0 and flags == 1  # ERR_TIMEOUT
    g = sv.SparseState(6)
    g.apply_gate((0,), np.array([[1, 1], [1, -1]]) / np.sqrt(2))
    assert g.num_terms() == 2
