"""Host-side logic of the learned propagator (no GPU): the parameter vector's
layout against the oracle's tensors, the seeded initialisation, and the
training examples drawn from a snapshot sequence."""
import numpy as np

from oracle import propagator as P
from paper_1310_2041_gb300 import hpf, learned


def test_pack_unpack_round_trip_in_oracle_layout():
    params = P.init_params(7)
    vec = hpf.pack_params(params)
    assert vec.dtype == np.float32 and vec.size == 9538
    # the documented layout: per layer W [27][C_in][C_out] then b [C_out]
    k = 0
    for (W, b), (ci, co, _) in zip(params, P.LAYERS):
        assert W.shape == (27, ci, co)
        np.testing.assert_array_equal(vec[k:k + W.size], W.astype(np.float32).ravel())
        k += W.size
        np.testing.assert_array_equal(vec[k:k + co], b.astype(np.float32))
        k += co
    assert k == vec.size
    back = hpf.unpack_params(vec)
    for (W, b), (W2, b2) in zip(params, back):
        np.testing.assert_array_equal(W.astype(np.float32), W2)
        np.testing.assert_array_equal(b.astype(np.float32), b2)


def test_init_params_is_seeded_he_uniform():
    a, b = learned.init_params(3), learned.init_params(3)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, learned.init_params(4))
    layers = hpf.unpack_params(a)
    for k, ((W, bias), (ci, co, _)) in enumerate(zip(layers, P.LAYERS)):
        bound = np.sqrt(6.0 / (27 * ci)) * (0.1 if k == 2 else 1.0)
        assert np.all(np.abs(W) <= bound) and np.all(bias == 0)
        # uniform on [-bound, bound]: the second moment is bound^2 / 3
        assert abs(np.mean(W.astype(np.float64) ** 2) / (bound ** 2 / 3) - 1) < 0.1


def test_training_examples_are_consecutive_triples():
    assert learned.triples(5) == [1, 2, 3]
    assert learned.triples(2) == []
