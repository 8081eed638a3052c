"""The seeded generator: host and device (torch) paths draw the same observation."""
import numpy as np

from paper_2412_10072_gb300 import synth


def test_device_path_reproduces_host_generator_noise_free():
    kw = dict(seed=3, n_ant=6, n_time=5, n_chan=12, flag_row_frac=0.2, n_src=7)
    host = synth.plain_large(noise=0.0, **kw)
    su = synth.plain_large_setup(**kw)
    dev = synth.make_observation_device(su, noise=0.0, noise_seed=0, device="cpu", rows_per_chunk=7)
    assert np.array_equal(dev["ant1"], host.ant1) and np.array_equal(dev["time_idx"], host.time_idx)
    assert np.array_equal(dev["flag"].numpy(), host.flag)
    scale = np.max(np.abs(host.data))
    assert np.max(np.abs(dev["data"].numpy() - host.data)) < 1e-6 * scale
    assert np.max(np.abs(dev["model"].numpy() - host.model)) < 1e-6 * scale


def test_noise_statistics_of_device_path():
    su = synth.plain_large_setup(seed=4, n_ant=5, n_time=40, n_chan=16, flag_row_frac=0.0, n_src=3)
    a = synth.make_observation_device(su, noise=0.0, noise_seed=1, device="cpu")
    su = synth.plain_large_setup(seed=4, n_ant=5, n_time=40, n_chan=16, flag_row_frac=0.0, n_src=3)
    b = synth.make_observation_device(su, noise=0.05, noise_seed=1, device="cpu")
    d = (b["data"] - a["data"]).numpy()
    assert abs(d.real.std() - 0.05) < 0.003 and abs(d.imag.std() - 0.05) < 0.003
