"""The BF16-emulating evaluation of the propagator oracle (tests/prop_bf16.py)
that the GPU network tests compare against, checked on the CPU: its rounding
against PyTorch's float32 -> bfloat16 conversion, and with nothing left to
round it is the oracle itself."""
import numpy as np
import torch

import prop_bf16 as E
from oracle import propagator as P


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -9, 65504.0]])
    a = a.astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(E.bf16(a), ref.astype(np.float64))


def test_emulation_without_rounding_effects_is_the_oracle():
    """Weights, inputs and (through a zero middle layer) the hidden values
    exact in BF16: the emulated forward equals the FP64 oracle to rounding."""
    rng = np.random.default_rng(1)
    params = [(E.bf16(W), np.zeros_like(b)) for W, b in P.init_params(2)]
    params[1] = (np.zeros_like(params[1][0]), np.zeros(16))   # h2 = SiLU(0) = 0 exactly
    x = E.bf16(rng.uniform(0.0, 1.0, size=(4, 5, 4, 6)))
    x[:2] = x[2:]                                             # zero change channels
    ye, _, _, _ = E.forward(params, x)
    yo, _ = P.forward(params, x)
    np.testing.assert_allclose(ye, yo, rtol=0, atol=1e-12)


def test_emulated_backward_tracks_the_oracle():
    """Inputs and weights exact in BF16: the emulated loss and weight
    gradients differ from the FP64 oracle's only by the hidden values' and
    gradients' BF16 roundings."""
    rng = np.random.default_rng(3)
    params = [(E.bf16(W * 0.5), E.bf16(rng.normal(scale=0.1, size=b.shape)).astype(np.float32)
               .astype(np.float64)) for W, b in P.init_params(4)]
    x = E.bf16(rng.uniform(0.0, 1.0, size=(4, 4, 3, 5)))
    nxt = E.bf16(rng.uniform(0.0, 1.0, size=(2, 4, 3, 5)))
    Le, ge = E.backward(params, x, nxt)
    Lo, go = P.backward(params, x, nxt - x[2:])
    # only BF16 roundings of hidden values and gradients separate the two
    assert abs(Le - Lo) <= 2e-2 * Lo
    for (a, _), (b, _) in zip(ge, go):
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b)
