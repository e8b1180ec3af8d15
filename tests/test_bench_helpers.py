"""CPU checks of the benchmark's work accounting (no GPU): the key-switch
work model against the figures derived by hand for the paper-shaped basis,
and the CPU-baseline extrapolation against a hand-computed sum."""
import bench


def test_keyswitch_work_matches_hand_counts():
    # level 24, K = alpha = 8, three digits: ModUp 24 inverse + 3 x 24 forward,
    # ModDown 16 inverse + 48 forward = 160 limb transforms per switch
    w = bench.keyswitch_work(16, 24, 8, 8)
    assert w["ks_limb_transforms"] == 160
    # plus the rescale: 2 inverse + 46 forward
    assert w["limb_transforms"] == 160 + 48
    assert w["butterflies"] == w["limb_transforms"] * (1 << 15) * 16
    # keys: 2 polys x 3 digits x 32 limbs of 2^16 words
    assert w["key_bytes"] == 2 * 3 * 32 * 8 * (1 << 16)
    # level 5, one digit, 8 special primes: 5 + 8 + 16 + 10 = 39
    assert bench.keyswitch_work(16, 5, 8, 8)["ks_limb_transforms"] == 39


def test_extrapolation_uses_each_levels_sample():
    W = dict(logN=16, n=245, d=5, k=256)  # one batch
    s = dict(alpha=8, ks_k=[0] + [2] * 30, t_ks={4: 1.0, 10: 2.0}, t_tensor4=0.5, t_enc4=0.25)
    hist = [0] * 31
    hist[4], hist[10], hist[5] = 3, 2, 1
    # level 5 borrows level 4's sample scaled by work 1 x (5 + 2) / (4 + 2)
    want = 3 * 1.0 + 2 * 2.0 + 1 * 1.0 * 7 / 6
    want += 1 * (0.25 * 6 / 4 + 5 * 0.5 * (6 / 4 + 1))
    assert abs(bench.extrapolate(s, hist, W, factored=True) - want) < 1e-12
