"""The autotuner's persistent cache (FH_AUTOTUNE_CACHE).

fh_autotune keeps each grid shape's fastest launch shape (tile width, block
warps, direction pairs on or off, item schedule) in a JSON file when FH_AUTOTUNE_CACHE names one; a later
process reads it and takes the cached shape without timing.  Checked on the
GPU with fresh processes: the shape a first process chose is reused by a
second one, a hand-written entry is taken as given, and both searches equal
the CPU oracle.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys, time
sys.path.insert(0, %(root)r)
import numpy as np, torch
import oracle
from paper_1407_8333_gb300 import build, fh, synth
build.build(); fh.load()
nd = %(n_dir)d
inp, pp = synth.random_case(303, n_fft=40, n_bins=300, n_fdot=70, n_dir=nd, p=0.3)
dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
plan = fh.fh_create_plan(fh.make_desc(pp, 40, nd, inp.n_peaks))
fh.fh_correct_doppler(plan, *dev)
t0 = time.perf_counter()
tile, warps = fh.fh_autotune(plan, 0, nd)
dt = time.perf_counter() - t0
fh.fh_transform(plan, 0, nd)
cand = fh.fh_select_candidates(plan, 0, nd)
fh.fh_destroy_plan(plan)
o = oracle.search(inp, pp)
c = cand.reshape(nd, -1, pp["top_k"])
ok = all(np.array_equal(c[k], o[k]) for k in ("cell", "row", "count"))
print(json.dumps({"tile": tile, "warps": warps, "seconds": dt, "oracle_equal": bool(ok),
                  "gpu": torch.cuda.get_device_name(0).replace(" ", "_"),
                  "n_f0": pp["n_f0"], "n_fdot": pp["n_fdot"], "k": pp["k_over"],
                  "t_fft": pp["t_fft"]}))
'''


def _child(cache, n_dir=2):
    env = dict(os.environ, FH_AUTOTUNE_CACHE=cache)
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT, "n_dir": n_dir}], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_second_process_reuses_the_cached_shape(tmp_path):
    cache = str(tmp_path / "autotune.json")
    first = _child(cache)
    assert first["oracle_equal"]
    entries = json.load(open(cache))["entries"]
    assert len(entries) == 1 and entries[0]["tile_cells"] == first["tile"]
    assert entries[0]["item_counter"] in (0, 1) and entries[0]["dir_pairs"] in (0, 1)
    second = _child(cache)
    assert second["oracle_equal"]
    assert (second["tile"], second["warps"]) == (first["tile"], first["warps"])


@pytest.mark.parametrize("n_dir", [2, 1])
def test_a_written_entry_is_taken_as_given(tmp_path, n_dir):
    cache = str(tmp_path / "autotune.json")
    probe = _child(cache, n_dir)
    key = ("%s|mode2|w0|n_f0=%d|n_fdot=%d|K=%d|T=%.17g|n_fft=40|n_dir=%d"
           % (probe["gpu"], probe["n_f0"], probe["n_fdot"], probe["k"], probe["t_fft"], n_dir))
    # every written shape is taken as given and searches like the oracle: no
    # pairs with the item counter, pairs (two directions, or one direction's
    # row halves) with every grid-th item
    for pairs, counter in ((0, 1), (1, 0)):
        with open(cache, "w") as f:
            f.write('{"version": 1, "entries": [\n{"key": "%s", "tile_cells": 512, '
                    '"block_warps": 20, "dir_pairs": %d, "item_counter": %d, "ms": 0}\n]}\n'
                    % (key, pairs, counter))
        got = _child(cache, n_dir)
        assert (got["tile"], got["warps"]) == (512, 20)
        assert got["oracle_equal"]
