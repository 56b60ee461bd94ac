"""CPU checks of the exact spectral Taylor-Green generator (inputs.taylor_green_spectral).

Its coefficients are written out by hand from sin/cos in exponential form; they must equal
the oracle's forward transform of the Taylor-Green velocity sampled on the mesh (the
library FFT, pinned elsewhere against the triple-sum DFT), and every other mode must be
exactly zero (so a state set from it vanishes outside the 2/3 box).
"""

import numpy as np
import pytest
import torch

from oracle import spectral_ns as sn
from paper_1602_03638_gb300 import inputs


@pytest.mark.parametrize("N", [4, 8, 12, 32])
def test_taylor_green_spectral_is_the_transform_of_the_mesh_field(N):
    got = inputs.taylor_green_spectral(N).numpy()
    ref = sn.to_spectral(inputs.taylor_green(N))
    assert got.shape == ref.shape == (3, N, N, N // 2 + 1)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * N ** 3)


def test_taylor_green_spectral_has_eight_modes_and_exact_zeros():
    uh = inputs.taylor_green_spectral(16)
    nz = torch.nonzero(uh)
    assert len(nz) == 8  # u and v at (+-1, +-1, kz = 1)
    assert set(int(k) for k in nz[:, 3]) == {1} and set(int(c) for c in nz[:, 0]) == {0, 1}
    assert torch.all(uh[2] == 0)
    c = inputs.taylor_green_spectral(8, dtype=torch.complex64)
    assert c.dtype == torch.complex64 and abs(complex(c[0, 1, 1, 1]) - (-1j * 64.0)) == 0.0
