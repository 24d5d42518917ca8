"""The seeded inputs of the paper's own glass model (Sec. 2.2), checked
against closed forms: sigma_SS = 2 sin(pi/10) = (sqrt 5 - 1) / 2,
sigma_LL = 2 sin(pi/5) = sqrt((5 - sqrt 5) / 2), N_L / N_S = (1 + sqrt 5) / 4
(N = 400: 221 small and 179 large discs), number density 1."""
import math

import numpy as np


def test_paper_sl_model(syn):
    assert abs(syn.SL_SIGMA[0, 0] - (math.sqrt(5.0) - 1.0) / 2.0) < 1e-15
    assert abs(syn.SL_SIGMA[1, 1] - math.sqrt((5.0 - math.sqrt(5.0)) / 2.0)) < 1e-15
    assert syn.SL_SIGMA[0, 1] == syn.SL_SIGMA[1, 0] == 1.0
    assert np.array_equal(syn.SL_EPS, [[0.5, 0.5], [0.5, 1.0]])
    x, t, H = syn.random_glass_start(400, 2, 0, fraction_a=syn.SL_FRACTION_S,
                                     density=syn.SL_DENSITY)
    assert (t == 0).sum() == 221 and (t == 1).sum() == 179
    assert np.allclose(H, np.eye(2) * 20.0)
    assert x.min() >= 0.0 and x.max() < 20.0


def test_splitmix64_matches_its_published_sequence(syn):
    """The counter-based stream is SplitMix64 (Steele, Lea, Flood 2014; Vigna's
    reference code) with state key * 0xD1B54A32D192ED03 + (k + 1) * golden
    gamma: choosing the key whose scrambled state is 1234567 must give the
    reference generator's first outputs for seed 1234567."""
    G2 = 0xD1B54A32D192ED03
    key = (1234567 * pow(G2, -1, 2 ** 64)) % 2 ** 64
    out = [int(v) for v in syn.splitmix64(key, np.arange(5, dtype=np.uint64))]
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]
    # uniform doubles use the top 53 bits
    u = syn.uniform(key, 2)
    assert u[0] == (6457827717110365317 >> 11) / 2.0 ** 53
    assert u[1] == (3203168211198807973 >> 11) / 2.0 ** 53
