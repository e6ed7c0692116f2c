"""The rate probes behind the clock-normalised roofline (ccc_mma_rate, ccc_popc_rate).

Each MMA probe fills its operands with 1.0 of its kind (and the block-scaled
kinds' scale factors with 1.0), so every accumulator entry must come out as
n_mma x K: that checks the operand encoding, the instruction descriptor and
the unit scale factors that the FP4 tally path relies on.
"""

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


@pytest.mark.parametrize("n_cols", [128, 224, 240, 256])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_mma_probe_accumulators_exact(kind, n_cols):
    import paper_1705_08213_gb300 as ccc
    cycles, bad = ccc.ccc_mma_rate(kind, n_cols=n_cols, n_mma=1000, clusters=3)
    assert bad == 0
    assert len(cycles) == 3 and all(c > 0 for c in cycles)


def test_mma_probe_rejects_bad_arguments():
    import torch

    import paper_1705_08213_gb300 as ccc
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for args in ((3, 256, 10, 1), (0, 200, 10, 1), (0, 272, 10, 1), (0, 48, 10, 1), (0, 256, 0, 1), (0, 256, 65537, 1),
                 (0, 256, 10, sms // 2 + 1)):
        with pytest.raises(ccc.CCCError) as e:
            ccc.ccc_mma_rate(*args)
        assert e.value.status == ccc.CCC_EINVAL


def test_popc_probe_runs():
    import paper_1705_08213_gb300 as ccc
    cycles = ccc.ccc_popc_rate(iters=256, blocks=4)
    assert len(cycles) == 4 and all(c > 0 for c in cycles)
