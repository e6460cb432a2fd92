"""Host-side argument checks of the Python API (no GPU needed)."""
import pytest

from paper_2503_17491_gb300 import api


@pytest.mark.parametrize("window", [0, 5])
def test_mapper_window_must_fit_the_views(window):
    with pytest.raises(ValueError):
        api.Mapper(capacity=10, max_views=4, max_pixels=100, n_new=1, max_keyframes=window)
