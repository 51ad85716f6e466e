"""Pins of the oracle's RFI mitigation (Sec. "AMBER", "RFI mitigation
(optional)"; three iterations of a time-domain filter for bright wide-band
low-DM RFI and of a frequency-domain filter for narrowband RFI) on inputs
built with known answers."""
import numpy as np

import oracle
import synth

T = synth.ARTS_T_SAMP_S


def test_clean_noise_is_untouched():
    x = synth.filterbank(2, 2, 128, 3000)
    y, tf, cf = oracle.rfi_clean(x, time_thresh=6.0, freq_thresh=6.0)
    assert tf.sum() == 0 and cf.sum() == 0
    assert (y == x).all()


def test_broadband_spike_is_replaced_by_channel_means():
    x = synth.filterbank(3, 1, 256, 4000)
    x[0, :, 1234] = np.minimum(255, x[0, :, 1234].astype(int) + 60)
    y, tf, cf = oracle.rfi_clean(x, time_thresh=5.0, freq_thresh=0.0)
    assert np.nonzero(tf[0])[0].tolist() == [1234]
    keep = np.ones(4000, bool)
    keep[1234] = False
    means = x[0][:, keep].astype(np.int64).sum(1)
    want = (2 * means + keep.sum()) // (2 * keep.sum())      # rounded half up
    assert (y[0, :, 1234] == want).all()
    assert (np.delete(y[0], 1234, axis=1) == np.delete(x[0], 1234, axis=1)).all()


def test_iterations_unmask_weaker_rfi():
    # a very bright spike inflates sigma so a weaker one hides in the first iteration
    x = synth.filterbank(4, 1, 256, 4000)
    x[0, :, 500] = np.minimum(255, x[0, :, 500].astype(int) + 120)
    x[0, :, 2500] = np.minimum(255, x[0, :, 2500].astype(int) + 5)   # ~ 5 sigma of the zero-DM series
    _, tf1, _ = oracle.rfi_clean(x, time_thresh=4.0, time_iters=1, freq_thresh=0.0)
    _, tf3, _ = oracle.rfi_clean(x, time_thresh=4.0, time_iters=3, freq_thresh=0.0)
    assert tf1[0, 500] == 1 and tf1[0, 2500] == 0
    assert tf3[0, 500] == 1 and tf3[0, 2500] == 1


def test_narrowband_and_dead_channels():
    x = synth.filterbank(5, 2, 128, 3000)
    x[0, 40] = np.minimum(255, x[0, 40].astype(int) + 25)   # persistent narrowband RFI
    x[1, 7] = 0                                              # dead channel
    y, tf, cf = oracle.rfi_clean(x, time_thresh=0.0, freq_thresh=5.0)
    assert np.nonzero(cf[0])[0].tolist() == [40] and np.nonzero(cf[1])[0].tolist() == [7]
    for tab, c in ((0, 40), (1, 7)):
        keep = np.ones(128, bool)
        keep[c] = False
        level = (2 * x[tab][keep].astype(np.int64).sum() + keep.sum() * 3000) // (2 * keep.sum() * 3000)
        assert (y[tab, c] == level).all()
        assert (np.delete(y[tab], c, axis=0) == np.delete(x[tab], c, axis=0)).all()


def test_dispersed_pulse_survives():
    f = synth.channel_freqs(256)
    x = synth.filterbank(6, 1, 256, 6000, pulses=[dict(tab=0, start=1000 + oracle.delays(f, T, 300.0, 1.0, 1)[0],
                                                       width=4, amp=synth.pulse_amplitude(40.0, 256, 4))])
    y, tf, cf = oracle.rfi_clean(x, time_thresh=4.5, freq_thresh=4.5)
    assert tf.sum() == 0 and cf.sum() == 0 and (y == x).all()
