"""ASPC density predictor (qmmm_aspc_predict) against the oracle's weights."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nhist", [1, 2, 4, 7])
def test_aspc_matches_oracle(nhist):
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    rng = np.random.default_rng(nhist)
    hist = [rng.normal(size=(37, 41)) for _ in range(nhist)]
    out = q.qmmm_aspc_predict([torch.as_tensor(h, device="cuda") for h in hist])
    torch.cuda.synchronize()
    ref = oracle.aspc_predict(hist)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-13 * np.max(np.abs(ref))


def test_aspc_rejects_host_memory_and_bad_sizes():
    import paper_2408_03273_gb300 as q
    torch = pytest.importorskip("torch")
    with pytest.raises(q.QMMMError):
        q.qmmm_aspc_predict([torch.zeros(4, dtype=torch.float64)])  # host tensor
    with pytest.raises(q.QMMMError):
        q.qmmm_aspc_predict([torch.zeros(4, dtype=torch.float64, device="cuda")] * 10)  # nhist > 9
