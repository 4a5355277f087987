"""GPU parity of the range-Doppler maps (gh_make_maps) and the measurement
synthesiser (gh_synth) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import maps as omaps
from oracle import model
from paper_2307_16550_gb300 import scenes
from tests.helpers import measurement64, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL_MAP = 1e-5  # float32 FFT, relative to the map's largest bin


def _scene(kind, seed=1):
    if kind == "tiny":
        return scenes.tiny_scene(seed)
    if kind == "paper":
        return scenes.paper_frame(seed)
    Ms, Mc, pad = {"small_pad2": (16, 8, 2), "pad1": (32, 16, 1), "pad8": (8, 16, 8), "big": (512, 256, 4)}[kind]
    radar = scenes.Radar(24e9, 250e6, 128e-6, Ms, Mc, pad)
    grid = scenes.Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), (4, 4, 2, 2))
    return scenes.custom_scene(seed, radar, grid, Q=3, T=2, snr_db=10.0)


@pytest.mark.parametrize("kind", ["tiny", "paper", "small_pad2", "pad1", "pad8", "big"])
def test_maps_match_oracle(ctx, torch_cuda, kind):
    sc = _scene(kind)
    Y32, Y = measurement64(sc)
    ref = omaps.centred_maps(Y, sc.radar.pad)
    got = ctx.maps(sc.radar, to_dev(torch_cuda, Y32)).cpu().numpy()
    assert got.shape == ref.shape
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < TOL_MAP, err


def test_maps_of_pure_tone_peak(ctx, torch_cuda):
    """On-bin tone of unit amplitude: centred bin value has modulus Ms*Mc."""
    Ms, Mc, pad = 64, 32, 4
    i0, j0 = 77, 45
    mc = np.arange(Mc)[:, None]
    m = np.arange(Ms)[None, :]
    Y = np.exp(2j * np.pi * (j0 / (pad * Mc) * mc + i0 / (pad * Ms) * m)).astype(np.complex64)[None]
    radar = scenes.Radar(24e9, 250e6, 1e-4, Ms, Mc, pad)
    got = ctx.maps(radar, to_dev(torch_cuda, Y)).cpu().numpy()[0]
    assert abs(abs(got[i0, j0]) - Ms * Mc) < 1e-3 * Ms * Mc
    assert np.unravel_index(np.argmax(np.abs(got)), got.shape) == (i0, j0)


@pytest.mark.parametrize("kind", ["tiny", "paper"])
def test_synth_matches_oracle_measurement(ctx, torch_cuda, kind):
    sc = _scene(kind, seed=3)
    ref = model.measurement(sc)
    noise = to_dev(torch_cuda, sc.noise.astype(np.complex64))
    got = ctx.synth(sc.radar, sc.tx, sc.rx, sc.targets, sc.alpha, noise).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()


def test_synth_without_noise_or_targets(ctx, torch_cuda):
    sc = scenes.tiny_scene(2)
    Y = ctx.synth(sc.radar, sc.tx, sc.rx, np.zeros((0, 4)), np.zeros((0, 3)), None).cpu().numpy()
    assert np.all(Y == 0)
