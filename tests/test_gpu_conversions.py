"""The FP64 kernels convert between binary64 and binary32 on the integer
pipe (the hardware conversion instructions share the narrow FP64 pipe of
this GPU).  Those conversions must equal the hardware's bit for bit:
round to nearest with ties to even for binary64 -> binary32 (IEEE 754
Sec. 4.3.1), exact widening binary32 -> binary64.  The batched residual's fixed-point map (nearest multiple of
2^(E-1080), ties away from zero) must equal exact FP64 scaling, floor and
the tie rule."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_conversions_match_hardware():
    import paper_1708_08434_gb300 as pkg
    for seed in (0x5EED, 12345):
        bad = pkg.check_conversions(1 << 26, seed)
        assert bad == (0, 0, 0), (seed, bad)
