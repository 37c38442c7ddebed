"""CPU model of the keys merge pass's tile geometry, checked over many sizes.

It restates the integer arithmetic of the persistent merge kernel in
csrc/nsort.cu and csrc/sort_device.cuh:
- the pair-aligned tiling (pair_tiles);
- each tile's slices from its two splitters, clamped to the runs
  (pair_tile_from, clamp_coranks);
- where the slices sit in the shared-memory buffer (smem_slices);
- the bulk-copy windows rounded out to 16 bytes and clipped at the last
  16-byte boundary of the array (issue_tile);
- the warps' loads of the few elements past that boundary;
- the 32 largest-key sentinels behind each slice;
- each thread's merge-path split (merge_path_plain) and its unchecked serial
  merge (serial_merge_sentinel).

For every tile it checks the following, and compares each pass's output with
numpy's sort of the pass's runs:
- every bulk copy starts on a 16-byte boundary inside the array;
- no write lands outside the kernel's buffer, and the two slices do not
  overlap;
- every shared-memory read hits an element or a sentinel that was written.

Run lengths are deliberately odd (the library's are multiples of the tile
sort's 16384 or 4096 keys), so that slices start at every alignment.  A change
to the kernel's geometry must be mirrored here."""
import numpy as np
import pytest

SENT = 32


def merge_path(a, b, diag):
    lo, hi = max(0, diag - len(b)), min(diag, len(a))
    while lo < hi:
        mid = (lo + hi) >> 1
        if a[mid] <= b[diag - 1 - mid]:
            lo = mid + 1
        else:
            hi = mid
    return lo


def merge_pass(x, run, NT, VT, word_bytes, top):
    """One merge pass of runs of `run` keys over x, as the kernel does it;
    returns the output array."""
    n = x.size
    TILE = NT * VT
    EPV = 16 // word_bytes
    IN_LEN = (TILE + 2 * SENT + 16) & ~3
    n_al = n & ~(EPV - 1)
    tpp = -(-2 * run // TILE)
    full, rem = n // (2 * run), n - (n // (2 * run)) * 2 * run
    tiles = full * tpp + -(-rem // TILE)

    def pair_of(t):
        pair, j = divmod(t, tpp)
        pair0 = pair * 2 * run
        la = min(run, n - pair0)
        rest = n - pair0 - run
        lb = 0 if rest <= 0 else min(rest, run)
        return j, pair0, la, lb

    split = []
    for t in range(tiles):
        j, pair0, la, lb = pair_of(t)
        split.append(merge_path(x[pair0:pair0 + la], x[pair0 + la:pair0 + la + lb], j * TILE))
    y = np.full(n, -1, dtype=np.int64)
    for t in range(tiles):
        j, pair0, la, lb = pair_of(t)
        pend = pair0 + la + lb
        out0 = pair0 + j * TILE
        out1 = min(out0 + TILE, pend)
        a_beg = split[t]
        a_end = la if out1 == pend else split[t + 1]
        # clamp_coranks
        d0, d1 = out0 - pair0, out1 - pair0
        a_beg = min(max(a_beg, max(0, d0 - lb)), min(d0, la))
        a_end = min(max(a_end, max(d1 - lb, a_beg)), min(a_beg + (d1 - d0), la))
        na, count = a_end - a_beg, out1 - out0
        nb = count - na
        a_off, b_off = pair0 + a_beg, pair0 + la + (d0 - a_beg)
        # smem_slices
        sh_a = a_off & (EPV - 1)
        base_b = (sh_a + na + SENT + EPV - 1) & ~(EPV - 1)
        sh_b = b_off & (EPV - 1)
        a0, b0 = sh_a, base_b + sh_b
        s = np.full(IN_LEN, -7, dtype=np.int64)            # -7: never written
        # issue_tile: windows rounded out to 16 bytes, clipped at n_al
        aw0, aw1 = a_off & ~(EPV - 1), min((a_off + na + EPV - 1) & ~(EPV - 1), n_al)
        bw0, bw1 = b_off & ~(EPV - 1), min((b_off + nb + EPV - 1) & ~(EPV - 1), n_al)
        if na > 0 and aw1 > aw0:
            assert aw0 % EPV == 0 and 0 <= aw0 and aw1 <= n
            assert aw1 - aw0 <= base_b                       # A's copy ends before B's window
            s[0:aw1 - aw0] = x[aw0:aw1]
        if nb > 0 and bw1 > bw0:
            assert bw0 % EPV == 0 and 0 <= bw0 and bw1 <= n and base_b % EPV == 0
            assert base_b + (bw1 - bw0) <= IN_LEN
            s[base_b:base_b + (bw1 - bw0)] = x[bw0:bw1]
        # the warps' own loads past n_al (at most EPV - 1 per slice)
        if a_off + na > n_al or b_off + nb > n_al:
            for i in range(max(a_off, n_al), a_off + na):
                assert i - max(a_off, n_al) < EPV - 1
                s[a0 + i - a_off] = x[i]
            for i in range(max(b_off, n_al), b_off + nb):
                assert i - max(b_off, n_al) < EPV - 1
                s[b0 + i - b_off] = x[i]
        # sentinels behind each slice
        assert a0 + na + SENT <= base_b and b0 + nb + SENT <= IN_LEN
        s[a0 + na:a0 + na + SENT] = top
        s[b0 + nb:b0 + nb + SENT] = top
        assert np.all(s[a0:a0 + na] == x[a_off:a_off + na])
        assert np.all(s[b0:b0 + nb] == x[b_off:b_off + nb])
        for tid in range(NT):
            diag = min(tid * VT, count)
            lo, hi = max(0, diag - nb), min(diag, na)
            while lo < hi:
                mid = (lo + hi) >> 1
                if s[a0 + mid] <= s[b0 + diag - 1 - mid]:
                    lo = mid + 1
                else:
                    hi = mid
            a, b = a0 + lo, b0 + diag - lo
            ka, kb = s[a], s[b]
            for k in range(VT):
                take_a = ka <= kb
                o = ka if take_a else kb
                nx = (a if take_a else b) + 1
                assert nx < IN_LEN and s[nx] != -7, "read of an unwritten word"
                if take_a:
                    a, ka = nx, s[nx]
                else:
                    b, kb = nx, s[nx]
                if tid * VT + k < count:
                    y[out0 + tid * VT + k] = o
    return y


@pytest.mark.parametrize("word_bytes,NT,VT", [(4, 128, 31), (8, 128, 15)])
@pytest.mark.parametrize("n,run", [(1, 1), (7, 3), (4001, 1000), (9999, 1331), (20_011, 5003),
                                   (4 * 3968 + 13, 2 * 3968 + 1), (12_345, 4096)])
def test_merge_pass_geometry(word_bytes, NT, VT, n, run):
    top = (1 << (8 * word_bytes - 1)) - 1       # the largest key (a signed model of all-ones)
    rng = np.random.default_rng(n * 31 + run)
    passes = 0
    for hi in (50, top):                          # heavy ties, and the largest key itself
        x = rng.integers(0, hi, size=n, dtype=np.int64, endpoint=True)
        r = run
        for s0 in range(0, n, r):
            x[s0:s0 + r] = np.sort(x[s0:s0 + r])
        while r < n:
            y = merge_pass(x, r, NT, VT, word_bytes, top)
            want = x.copy()
            for s0 in range(0, n, 2 * r):
                want[s0:s0 + 2 * r] = np.sort(x[s0:s0 + 2 * r])
            np.testing.assert_array_equal(y, want)
            x, r = y, 2 * r
            passes += 1
    assert passes == 2 * max(0, int(np.ceil(np.log2(n / run))))
