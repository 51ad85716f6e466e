"""CPU checks of the pattern-factored dedispersion kernel's shared-memory
addressing and arithmetic: the library's own host tables
(fdd_fact_tables_host) drive a numpy emulation of every block of the kernel
-- raw staging as the kernel's TMA copies do it (one unshifted row of Lw
words per channel into raw buffer s & 1, zeros past the row's valid words,
and arbitrary bytes between the last valid sample and the end of its word),
pattern-row builds (two aligned words joined by a funnel shift, even/odd
byte lanes, PRMT packing, the shifted copy with the neighbouring lane's
sample), and the per-trial accumulation -- which must stay inside each
shared-memory region (a build reads only the Lw words its channel's copy
wrote) and reproduce the oracle's brute-force series exactly."""
import numpy as np
import pytest

import oracle
import synth

T_SAMP = synth.ARTS_T_SAMP_S


def prmt(a, b, sel):
    """Byte permute of two uint32 arrays (selector nibbles pick bytes of b:a)."""
    a = np.asarray(a, np.uint64)
    b = np.asarray(b, np.uint64)
    src = (b << np.uint64(32)) | a
    out = np.zeros_like(a)
    for n in range(4):
        k = (sel >> (4 * n)) & 7
        out |= ((src >> np.uint64(8 * k)) & np.uint64(0xFF)) << np.uint64(8 * n)
    return out.astype(np.uint32)


class Smem:
    def __init__(self, n):
        self.m = np.full(n, 0xCD, np.uint8)

    def rd32(self, addr, lo, hi):
        addr = np.asarray(addr, np.int64)
        assert (addr >= lo).all() and (addr + 4 <= hi).all(), "read outside [%d, %d)" % (lo, hi)
        assert (addr % 4 == 0).all()
        b = self.m[addr[..., None] + np.arange(4)]
        return (b.astype(np.uint32) << (8 * np.arange(4, dtype=np.uint32))).sum(-1).astype(np.uint32)

    def wr32(self, addr, val, lo, hi):
        addr = np.asarray(addr, np.int64)
        assert (addr >= lo).all() and (addr + 4 <= hi).all(), "write outside [%d, %d)" % (lo, hi)
        assert (addr % 4 == 0).all()
        val = np.asarray(val, np.uint32)
        for k in range(4):
            self.m[addr + k] = ((val >> np.uint32(8 * k)) & np.uint32(0xFF)).astype(np.uint8)


def funnel_r(lo, hi, sh):
    """__funnelshift_r: low 32 bits of (hi:lo) >> (sh & 31)."""
    w = (np.asarray(hi, np.uint64) << np.uint64(32)) | np.asarray(lo, np.uint64)
    return ((w >> np.uint64(sh & 31)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def emulate(x, n_valid, sb_map, tb, v, CC, n_dm, n_out, E=1):
    """x: uint8 rows (E = 1) or the uint16 rows of a downsampled range (E = 2), n_valid samples."""
    G, BD, T = v["group"], v["dm_per_block"], v["tile"]
    NW = T // 64
    Lw, pat_bytes, smem_bytes = tb["Lw"], tb["pat_bytes"], tb["smem_bytes"]
    PB = tb["pat_bufs"]
    rb, raw_lo = tb["rb"], tb["raw_off"]
    n_chan = x.shape[1]
    gps = CC // G
    zero_lo, zero_hi = tb["zero_off"], tb["zero_off"] + 4 * Lw + 16
    assert zero_hi <= raw_lo and raw_lo % 128 == 0 and rb % 128 == 0 and rb >= 4 * Lw
    assert PB in (1, 2)
    raw_hi = raw_lo + 2 * CC * rb
    pat_lo, pat_hi = tb["pat_off"], tb["pat_off"] + PB * pat_bytes
    assert pat_lo == raw_hi
    goff_lo = pat_hi
    desc_lo = goff_lo + (PB + 1) * gps * BD * 4
    max_desc = int(tb["pd_idx"][..., 1].max())
    assert desc_lo + PB * max_desc * tb["desc_ints"] * 4 == tb["bar_off"] and tb["bar_off"] % 8 == 0
    assert tb["bar_off"] + 16 + 128 == smem_bytes       # mbarriers + base alignment slack
    assert desc_lo % 16 == 0 and max_desc * (tb["desc_ints"] // 4) <= v["threads"]
    words_valid = (n_valid * E + 3) // 4                 # the tensor's row length in words

    def pat_buf(s):
        """Pattern-row bytes stage s may write and read."""
        if PB == 1:
            return pat_lo, pat_hi
        lo = pat_lo + (s % 2) * pat_bytes
        return lo, lo + pat_bytes

    def slot_of(addr):
        """Bounds of the region a build read at addr may touch."""
        if addr < zero_hi:
            return zero_lo, zero_hi
        k = (addr - raw_lo) // rb
        return raw_lo + k * rb, raw_lo + k * rb + (rb if tb["box_rows"] > 1 else 4 * Lw)
    n_sb = sb_map.shape[0]
    S = np.zeros((n_sb, n_dm, n_out), np.int64)
    lanes = np.arange(32)
    n_stages = tb["n_stages"]
    for sb in range(n_sb):
        for blk in range(tb["n_blk"]):
            for tile in range((n_out + T - 1) // T):
                t0 = tile * T
                sm = Smem(smem_bytes)
                sm.m[zero_lo:zero_hi] = 0
                acc = np.zeros((BD, T), np.int64)

                def stage_raw(s):
                    c0 = s * CC
                    for cc in range(min(CC, n_chan - c0)):   # raw staging (the TMA box of stage s)
                        c = c0 + cc
                        if tb["box_rows"] > 1:
                            # the channel's row arrives in its channel box: rb bytes from the box's start
                            start = (t0 + tb["bbase"][blk, c // tb["box_rows"]]) * E
                            width = rb
                        else:
                            start = (t0 + tb["base"][blk, c]) * E  # byte of the row's first staged sample
                            width = 4 * Lw
                        assert start % 16 == 0                     # TMA x coordinate on a 16-byte boundary
                        idx = start + np.arange(width)
                        row = np.ascontiguousarray(x[sb_map[sb, c], c]).view(np.uint8)   # little-endian bytes
                        byts = np.where(idx < 4 * words_valid, row[np.minimum(idx, row.size - 1)], 0)
                        byts = np.where((idx >= n_valid * E) & (idx < 4 * words_valid), 0xE7, byts)  # pitch padding
                        slot = raw_lo + ((s % 2) * CC + cc) * rb
                        sm.m[slot:slot + width] = byts.astype(np.uint8)

                def build(s):
                    stage_raw(s)
                    lo_p, hi_p = pat_buf(s)
                    sm.m[lo_p:hi_p] = 0xAB        # stale pattern bytes from an earlier stage
                    first, n_desc = tb["pd_idx"][blk, s]
                    for d in tb["pdesc"][first:first + n_desc]:   # pattern-row builds
                        dst0, dst1, nw4 = int(d[0]), int(d[1]), int(d[2])
                        src = d[3:3 + G].astype(np.int64)
                        j = np.arange(nw4)
                        ev = np.zeros(nw4, np.uint32)
                        od = np.zeros(nw4, np.uint32)
                        for k in range(G):
                            lo, hi = slot_of(int(src[k]))
                            if src[k] >= zero_hi:                  # this stage's raw buffer
                                assert (int(src[k]) - raw_lo) // (CC * rb) == s % 2
                            if E == 1:
                                al = (int(src[k]) & ~3) + 4 * j
                                xw = funnel_r(sm.rd32(al, lo, hi), sm.rd32(al + 4, lo, hi), 8 * int(src[k]))
                                ev = (ev + prmt(xw, 0, 0x4240)).astype(np.uint32)
                                od = (od + prmt(xw, 0, 0x4341)).astype(np.uint32)
                            else:
                                # 16-bit samples: a unit is two words, summed in 16-bit lanes (no carry)
                                assert int(src[k]) % 2 == 0
                                al = (int(src[k]) & ~3) + 8 * j
                                w0, w1, w2 = (sm.rd32(al + 4 * q, lo, hi) for q in range(3))
                                ev = (ev + funnel_r(w0, w1, 8 * int(src[k]))).astype(np.uint32)   # [R0, R1]
                                od = (od + funnel_r(w1, w2, 8 * int(src[k]))).astype(np.uint32)   # [R2, R3]
                        if E == 1:
                            A = prmt(ev, od, 0x5410)
                            B = prmt(ev, od, 0x7632)
                            C = prmt(od, ev, 0x7610)
                        else:
                            A, B = ev, od
                            C = prmt(A, B, 0x5432)
                        A_next = np.append(A[1:], np.uint32(0))
                        D = prmt(B, A_next, 0x5432)
                        sm.wr32(dst0 + 8 * j, A, lo_p, hi_p)
                        sm.wr32(dst0 + 8 * j + 4, B, lo_p, hi_p)
                        sm.wr32(dst1 + 8 * j, C, lo_p, hi_p)
                        sm.wr32(dst1 + 8 * j + 4, D, lo_p, hi_p)

                def accumulate(s):
                    ngs = (min(CC, n_chan - s * CC) + G - 1) // G
                    go = tb["goff"][blk, s * gps:s * gps + ngs]
                    lo_p, hi_p = pat_buf(s)
                    for gl in range(ngs):
                        for jj in range(BD):
                            o = int(go[gl, jj])
                            addr = o + 4 * lanes[None, :] + 128 * np.arange(NW)[:, None]
                            wv = sm.rd32(addr, lo_p, hi_p)
                            lo16 = (wv & 0xFFFF).astype(np.int64)
                            hi16 = (wv >> 16).astype(np.int64)
                            tt = 2 * (lanes[None, :] + 32 * np.arange(NW)[:, None])
                            acc[jj, tt.ravel()] += lo16.ravel()
                            acc[jj, tt.ravel() + 1] += hi16.ravel()

                if PB == 1:
                    for s in range(n_stages):
                        build(s)
                        accumulate(s)
                else:
                    # the kernel's order: stage s + 1 is built before stage s's adds read their rows
                    build(0)
                    for s in range(n_stages):
                        if s + 1 < n_stages:
                            build(s + 1)
                        accumulate(s)
                for jj in range(BD):
                    i = blk * BD + jj
                    if i < n_dm:
                        nt = min(T, n_out - t0)
                        S[sb, i, t0:t0 + nt] = acc[jj, :nt]
    return S


def fact_variants():
    try:
        import paper_2205_12362_b300 as fdd
        return [v for v in fdd.variants() if v["kind"] == 1]
    except Exception:
        return []


@pytest.mark.parametrize("v", fact_variants(), ids=lambda v: "v%d_G%d_bd%d_t%d" % (
    v["index"], v["group"], v["dm_per_block"], v["tile"]))
@pytest.mark.parametrize("CC", [8, 16])
def test_factored_kernel_emulation(v, CC):
    import paper_2205_12362_b300 as fdd
    if CC % v["group"]:
        pytest.skip("stage size not a multiple of G")
    rng = np.random.default_rng(v["index"] + CC)
    n_tab, n_chan, n_sb, n_out = 2, 37, 2, 300
    f = synth.channel_freqs(n_chan)
    n_dm = v["dm_per_block"] + 5
    ranges = [dict(dm0=3.0, ddm=2.5, n_dm=n_dm, downsamp=1, widths=[1])]
    d = oracle.delays(f, T_SAMP, 3.0, 2.5, n_dm)
    n_in = n_out + int(d.max()) + 3
    x = rng.integers(0, 256, size=(n_tab, n_chan, synth.padded_pitch(n_in)), dtype=np.int64).astype(np.uint8)
    sb = rng.integers(0, n_tab, size=(n_sb, n_chan)).astype(np.int16)
    tb = fdd.fact_tables_host(n_tab, n_chan, n_sb, f, T_SAMP, ranges, sb, 0, v["index"], CC)
    assert tb["Lw"] > 0
    if int(tb["pd_idx"][..., 1].max()) * (tb["desc_ints"] // 4) > v["threads"]:
        pytest.skip("layout the library refuses (stage descriptors exceed one int4 per thread)")
    assert (tb["delays"] == d).all()
    S = emulate(x, n_in, sb, tb, v, CC, n_dm, n_out)
    want = oracle.dedisperse(oracle.downsample(x, 1, n_in=n_in), sb, d, n_out)
    assert (S == want).all()


@pytest.mark.parametrize("v", fact_variants(), ids=lambda v: "v%d_G%d_bd%d_t%d" % (
    v["index"], v["group"], v["dm_per_block"], v["tile"]))
@pytest.mark.parametrize("D", [2, 4])
def test_factored_kernel_emulation_16bit(v, D):
    """The same emulation for a downsampled range: the staged rows are the
    16-bit sums of D samples (byte offsets twice the sample offsets, a build
    unit two words summed in 16-bit lanes), against the oracle's brute-force
    dedispersion of the oracle's downsampled rows."""
    import paper_2205_12362_b300 as fdd
    CC = 8 if v["group"] <= 8 else 16
    rng = np.random.default_rng(v["index"] + D)
    n_tab, n_chan, n_sb, n_out = 2, 37, 2, 150
    f = synth.channel_freqs(n_chan)
    n_dm = v["dm_per_block"] + 5
    ranges = [dict(dm0=3.0, ddm=2.5 * D, n_dm=n_dm, downsamp=D, widths=[1])]
    d = oracle.delays(f, T_SAMP, 3.0, 2.5 * D, n_dm, D)
    n_in = (n_out + int(d.max()) + 3) * D
    x = rng.integers(0, 256, size=(n_tab, n_chan, synth.padded_pitch(n_in)), dtype=np.int64).astype(np.uint8)
    sb = rng.integers(0, n_tab, size=(n_sb, n_chan)).astype(np.int16)
    tb = fdd.fact_tables_host(n_tab, n_chan, n_sb, f, T_SAMP, ranges, sb, 0, v["index"], CC)
    if tb["Lw"] < 0:
        pytest.skip("staged rows of twice the bytes exceed the kernel's row limit for this tile")
    if int(tb["pd_idx"][..., 1].max()) * (tb["desc_ints"] // 4) > v["threads"]:
        pytest.skip("layout the library refuses (stage descriptors exceed one int4 per thread)")
    assert (tb["delays"] == d).all()
    y = oracle.downsample(x, D, n_in=n_in)                  # the range's rows (sums of D bytes)
    assert y.max() < 1 << 16
    n_y = n_in // D
    S = emulate(y.astype(np.uint16), n_y, sb, tb, v, CC, n_dm, n_out, E=2)   # staged as 16-bit samples
    want = oracle.dedisperse(y, sb, d, n_out)
    assert (S == want).all()


@pytest.mark.parametrize("v", fact_variants(), ids=lambda v: "v%d_G%d_bd%d_t%d" % (
    v["index"], v["group"], v["dm_per_block"], v["tile"]))
def test_factored_kernel_emulation_channel_boxes(v):
    """A one-TAB plan, where consecutive channels are consecutive tensor
    rows: the raw rows of 8 (or 4) channels travel as one TMA box from the
    least of their staged starts, each channel's data shifted in its slot by
    its start's distance to that one, as the descriptors record."""
    import paper_2205_12362_b300 as fdd
    CC = 16 if 16 % v["group"] == 0 else 8
    rng = np.random.default_rng(v["index"] + 7)
    n_chan, n_out = 61, 300
    f = synth.channel_freqs(n_chan)
    n_dm = v["dm_per_block"] + 5
    ranges = [dict(dm0=3.0, ddm=0.5, n_dm=n_dm, downsamp=1, widths=[1])]   # rows of at most 256 words
    d = oracle.delays(f, T_SAMP, 3.0, 0.5, n_dm)
    n_in = n_out + int(d.max()) + 3
    x = rng.integers(0, 256, size=(1, n_chan, synth.padded_pitch(n_in)), dtype=np.int64).astype(np.uint8)
    sb = np.zeros((1, n_chan), np.int16)
    tb = fdd.fact_tables_host(1, n_chan, 1, f, T_SAMP, ranges, sb, 0, v["index"], CC)
    if tb["Lw"] < 0 or int(tb["pd_idx"][..., 1].max()) * (tb["desc_ints"] // 4) > v["threads"]:
        pytest.skip("layout the library refuses")
    assert tb["box_rows"] in (4, 8)
    S = emulate(x, n_in, sb, tb, v, CC, n_dm, n_out)
    want = oracle.dedisperse(oracle.downsample(x, 1, n_in=n_in), sb, d, n_out)
    assert (S == want).all()


def test_factored_tables_share_patterns():
    """On the ARTS band the factored tables need far fewer pattern rows than
    trials x groups (the source of the kernel's saving)."""
    import paper_2205_12362_b300 as fdd
    v = [v for v in fact_variants() if v["group"] == 8 and v["dm_per_block"] == 64][0]
    f = synth.channel_freqs(1536)
    ranges = [dict(dm0=0.0, ddm=0.2, n_dm=256, downsamp=1, widths=[1])]
    tb = fdd.fact_tables_host(1, 1536, 1, f, T_SAMP, ranges, np.zeros((1, 1536)), 0, v["index"], 32)
    rows = tb["n_desc"]
    trial_group_pairs = tb["n_blk"] * tb["n_groups"] * v["dm_per_block"]
    assert rows < trial_group_pairs / 4
