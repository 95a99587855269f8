"""CPU model of the tensor-core BlindRotate's job streams (csrc/tc.cu, `chunk_of`,
`decode_e` and the digit jobs' index split), checked without a GPU.

The persistent kernel hands out product jobs and digit jobs from two global counters.
The tiles (or tile pairs) are split into `nchunks` chunks of nearly equal size (the first
units % nchunks chunks one larger), and both streams run all steps of one chunk before the
next.  The model restates that mapping and checks what the schedule needs:

* every job index names a distinct (unit, step, entry), and all of them are named;
* within a chunk the order is step-major, and chunks follow each other;
* digit and product streams use the same chunks, so the product jobs of (step i, tile t)
  and the digit jobs of (step i, tile t) sit in the same chunk at the same position;
* no job depends on a job later in either stream (E(i, t) on D(i, t); D(i + 1, t) on all
  E(i, t)), which with in-order hand-out keeps the schedule free of deadlock.
"""
import math

import pytest


def chunk_of(job, units, nchunks, per_unit):
    """(first unit, units in the chunk, offset within the chunk) of stream entry `job`."""
    base, extra = units // nchunks, units % nchunks
    big = extra * (base + 1) * per_unit
    if job < big:
        c = job // ((base + 1) * per_unit)
        rem = job - c * (base + 1) * per_unit
    else:
        c = extra + (job - big) // (base * per_unit)
        rem = job - big - (c - extra) * base * per_unit
    return c * base + min(c, extra), base + (1 if c < extra else 0), rem


def nchunks_for(units, e_per_tile, sms=148, waves=3.8):
    min_units = math.ceil(waves * sms / e_per_tile)
    return max(1, units // max(1, min_units))


def product_stream(units, n, e_per_tile, nchunks):
    """(step, unit, entry within the unit) of every product job, in stream order."""
    out = []
    for job in range(n * units * e_per_tile):
        u0, uc, rem = chunk_of(job, units, nchunks, n * e_per_tile)
        len_c = uc * e_per_tile
        pos = rem % len_c
        out.append((rem // len_c, u0 + pos // e_per_tile, pos % e_per_tile))
    return out


def digit_stream(tiles, n, nchunks, parts=16):
    """(step, tile, part) of every digit job, in stream order (one SM per tile)."""
    out = []
    for job in range(n * tiles * parts):
        t0, tc, rem = chunk_of(job, tiles, nchunks, n * parts)
        i = rem // (tc * parts)
        r = rem % (tc * parts)
        out.append((i, t0 + r // parts, r % parts))
    return out


@pytest.mark.parametrize("tiles,n,e", [(32, 7, 36), (33, 5, 36), (64, 4, 36), (32, 3, 54),
                                       (7, 6, 16), (1, 9, 36), (50, 3, 24)])
def test_streams_cover_every_job_once_in_chunk_then_step_order(tiles, n, e):
    nch = nchunks_for(tiles, e)
    assert 1 <= nch <= tiles
    ps = product_stream(tiles, n, e, nch)
    assert sorted(ps) == sorted((i, t, k) for i in range(n) for t in range(tiles) for k in range(e))
    ds = digit_stream(tiles, n, nch)
    assert sorted(ds) == sorted((i, t, p) for i in range(n) for t in range(tiles) for p in range(16))
    # chunks: sizes differ by at most one and cover the tiles in order
    sizes = [tiles // nch + (1 if c < tiles % nch else 0) for c in range(nch)]
    assert sum(sizes) == tiles and max(sizes) - min(sizes) <= 1
    bounds = [sum(sizes[:c]) for c in range(nch + 1)]

    def chunk(t):
        return next(c for c in range(nch) if bounds[c] <= t < bounds[c + 1])

    # order: chunk-major, then step-major inside a chunk, in both streams
    for stream in (ps, ds):
        keys = [(chunk(t), i) for i, t, _ in stream]
        assert keys == sorted(keys)


@pytest.mark.parametrize("tiles,n,e", [(32, 6, 36), (33, 4, 54), (17, 5, 24)])
def test_no_job_waits_for_a_later_job(tiles, n, e):
    """E(i, t) needs all 16 digit jobs D(i, t); D(i + 1, t) needs all e jobs E(i, t).  With
    both streams handed out in order, a job may only wait for jobs that come earlier in
    the interleaving the schedule allows: every dependency of a product job precedes, in
    the digit stream, the digit jobs that depend on that product job's step."""
    nch = nchunks_for(tiles, e)
    ps = product_stream(tiles, n, e, nch)
    ds = digit_stream(tiles, n, nch)
    d_pos = {}
    for k, (i, t, p) in enumerate(ds):
        d_pos.setdefault((i, t), []).append(k)
    e_pos = {}
    for k, (i, t, _) in enumerate(ps):
        e_pos.setdefault((i, t), []).append(k)
    for (i, t), ks in e_pos.items():
        # the last digit job E(i, t) waits for precedes the first digit job waiting for it
        if (i + 1, t) in d_pos:
            assert max(d_pos[(i, t)]) < min(d_pos[(i + 1, t)])
        # product jobs of a later step of the same tile come later in the product stream
        if (i + 1, t) in e_pos:
            assert max(ks) < min(e_pos[(i + 1, t)])


def test_bench_level_splits_into_two_chunks_of_16():
    """The bench's 4096-gate level at Karatsuba level 2 (32 tiles, 36 product jobs per tile
    and step) on 148 SMs: two chunks of 16 tiles, 3.9 waves of product jobs per step each."""
    assert nchunks_for(32, 36) == 2
    assert nchunks_for(16, 36) == 1
    assert nchunks_for(64, 36) == 4
