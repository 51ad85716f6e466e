"""Seeded synthetic inputs shaped like ARTS Stokes-I filterbank data.

This module only makes data: noise, injected pulses at caller-given
per-channel arrival samples, SB-to-TAB tables and channel frequencies.  It
holds none of the search method's arithmetic (no dispersion delays, no
dedispersion, no statistics), so the oracle and the CUDA path can both be fed
from it without sharing method code.

Shapes follow the paper's data description: 8-bit Stokes I per tied-array
beam, 1536 channels over 300 MHz (1220-1520 MHz for the 1370 MHz band), 81.92
us sampling, time the fastest index (Sec. "Dedicated ARTS TABF on Central
Uniboards", Sec. "Data formats"); 12 TABs per compound beam and 71 synthesized
beams (Sec. "Hierarchical beam forming").
"""
import numpy as np

ARTS_N_CHAN = 1536
ARTS_F_LO_MHZ = 1220.0
ARTS_F_HI_MHZ = 1520.0
ARTS_T_SAMP_S = 81.92e-6
ARTS_N_TAB = 12
ARTS_N_SB = 71
ARTS_CHUNK = 12500  # 1.024 s / 81.92 us


def channel_freqs(n_chan=ARTS_N_CHAN, f_lo=ARTS_F_LO_MHZ, f_hi=ARTS_F_HI_MHZ):
    """Channel centre frequencies in MHz, ascending: f_lo + (c + 1/2) * bw / n_chan."""
    return f_lo + (np.arange(n_chan, dtype=np.float64) + 0.5) * ((f_hi - f_lo) / n_chan)


def padded_pitch(n_samp, align=16):
    """Row pitch (elements) rounded up so every channel row starts 16-byte aligned."""
    return (int(n_samp) + align - 1) // align * align


def pulse_amplitude(snr, n_chan, width, sd=16.0):
    """Per-channel amplitude (counts) that gives a boxcar of `width` samples an
    ideal matched-filter S/N of `snr` summed over `n_chan` channels of noise `sd`."""
    return float(snr) * float(sd) / np.sqrt(float(n_chan) * float(width))


def filterbank(seed, n_tab, n_chan, n_samp, pitch=None, mean=128.0, sd=16.0, pulses=(),
               noise=True):
    """uint8[n_tab][n_chan][pitch] = clip(rint(mean + sd*N(0,1) + pulses), 0, 255).

    pulses: iterable of dicts with keys
      tab    -- TAB index the pulse is injected into
      start  -- int array [n_chan], first sample of the pulse in each channel
      width  -- pulse width in samples (boxcar)
      amp    -- counts added per sample and channel (float)
      chans  -- optional: channels (index array or boolean mask) that get the
                pulse; all channels if absent
    Samples in [n_samp, pitch) are zero.  The noise stream is Philox(seed),
    drawn TAB by TAB as float32 standard normals.
    """
    pitch = padded_pitch(n_samp) if pitch is None else int(pitch)
    if pitch < n_samp:
        raise ValueError("pitch < n_samp")
    out = np.zeros((n_tab, n_chan, pitch), dtype=np.uint8)
    rng = np.random.Generator(np.random.Philox(int(seed)))
    by_tab = {}
    for p in pulses:
        by_tab.setdefault(int(p["tab"]), []).append(p)
    for tab in range(n_tab):
        if noise:
            v = rng.standard_normal((n_chan, n_samp), dtype=np.float32)
            v *= np.float32(sd)
            v += np.float32(mean)
        else:
            v = np.full((n_chan, n_samp), np.float32(mean), dtype=np.float32)
        for p in by_tab.get(tab, []):
            start = np.asarray(p["start"], dtype=np.int64)
            w = int(p["width"])
            amp = np.float32(p["amp"])
            sel = np.ones(n_chan, dtype=bool)
            if p.get("chans") is not None:
                sel = np.zeros(n_chan, dtype=bool)
                sel[np.asarray(p["chans"])] = True
            for k in range(w):
                t = start + k
                ok = (t >= 0) & (t < n_samp) & sel
                c = np.nonzero(ok)[0]
                v[c, t[ok]] += amp
        np.rint(v, out=v)
        np.clip(v, 0, 255, out=v)
        out[tab, :, :n_samp] = v.astype(np.uint8)
    return out


def sb_map_piecewise(seed, n_sb, n_chan, n_tab, sub=16):
    """int32[n_sb][n_chan]: each SB takes, per block of `sub` channels, one TAB
    drawn uniformly from [0, n_tab) by Philox(seed) (a seeded stand-in for the
    frequency-dependent TAB switching of synthesized beams)."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    n_blk = (n_chan + sub - 1) // sub
    blk = rng.integers(0, n_tab, size=(n_sb, n_blk), dtype=np.int64)
    return np.repeat(blk, sub, axis=1)[:, :n_chan].astype(np.int32)


def random_pulses(seed, n, n_tab_pool, dm_lo, dm_hi, widths, snr_lo, snr_hi, t_lo, t_hi):
    """Seeded pulse parameters (DM, width, S/N, t0, tab) for injection; the
    caller turns DM into per-channel arrival samples with its own model."""
    rng = np.random.Generator(np.random.Philox(int(seed) + 7919))
    out = []
    for _ in range(int(n)):
        out.append(dict(dm=float(rng.uniform(dm_lo, dm_hi)),
                        width=int(rng.choice(np.asarray(widths))),
                        snr=float(rng.uniform(snr_lo, snr_hi)),
                        t0=int(rng.integers(t_lo, t_hi)),
                        tab=int(rng.choice(np.asarray(n_tab_pool)))))
    return out


def sb_pulses(sb_row, start, width, amp):
    """Pulse dicts (for filterbank) that put one pulse into every channel of
    the TAB that an SB selects there (sb_row: [n_chan] TAB per channel), so
    that SB receives the whole pulse: a source at that SB's position."""
    sb_row = np.asarray(sb_row)
    return [dict(tab=int(k), start=start, width=width, amp=amp, chans=np.nonzero(sb_row == k)[0])
            for k in np.unique(sb_row)]
