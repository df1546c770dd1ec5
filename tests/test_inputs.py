"""The seeded input generators: the device evaluation of the hidden-truth
stream equals the host one (the year-long assimilative runs use it)."""
import numpy as np
import pytest

import sft_inputs as I


@pytest.mark.parametrize("t_hours", [0.0, 13.0, 24.0 * 40.5])
def test_truth_torch_equals_truth(t_hours):
    pytest.importorskip("torch")
    st = I.ObservationStream(40, 96, seed=2, days=60)
    a = st.truth(t_hours)
    b = st.truth_torch(t_hours, device="cpu").numpy()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(st.mu(t_hours) - st.mu_torch(t_hours, device="cpu").numpy()).max() <= 1e-15
