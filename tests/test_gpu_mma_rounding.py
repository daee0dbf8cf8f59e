"""The tensor core's FP32 accumulation, as the split-BF16 kernels assume it (kind::f16, sm_103a).

Measured behaviour pinned here: after every MMA the FP32 sum is truncated toward zero, and the
products are aligned to the largest term keeping two bits below its last significant bit; a
product smaller than that is dropped.  This is why the BF16x6 kernels keep the small correction
products in an accumulator of their own."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_12132_gb300 as fd  # noqa: E402

U = 2.0 ** -23          # ulp(1)
U_BELOW = 2.0 ** -24    # ulp just below 1


@pytest.mark.parametrize("reps", [1, 8])
def test_tensor_core_accumulation_truncates(reps):
    o = fd.fdetd_probe_mma_rounding(reps).astype(np.float64)
    c0, c1 = o[:, 0], o[:, 1]
    assert c0[0] == 1.0                         # 1 + 0.75u in one MMA -> 1 (round to nearest: 1 + u)
    assert c0[1] == 1.0                         # +0.75u per chained MMA is lost every time
    assert c1[1] == 1.0 - 2 * U_BELOW * reps    # 1 - 0.75u per MMA, truncated toward zero each time
    assert c0[2] == -1.0 and c1[2] == -(1.0 - 2 * U_BELOW * reps)
    assert c0[3] == 1.0 + 3 * U                 # 1 + 3.75u -> 1 + 3u: quarter-ulp products kept, sum truncated
    assert c0[4] == 1.0                         # tie -> toward zero
    assert c0[6] == 0.0                         # 2^-30 below a cancelling pair of ones is dropped
    assert c0[7] == 0.0
    assert c0[8] == 1.0                         # eighth-ulp products are dropped one by one
    assert c0[9] == 1.0 + 4 * U * reps          # quarter-ulp products add up exactly inside one MMA
    assert c0[10] == 1.0 and c0[11] == 1.0
