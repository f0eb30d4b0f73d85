"""Resource guards on the compiled kernels (CPU: reads the ptxas report that
the build writes).  Local memory in a hot kernel is a silent slowdown: a
runtime index into a per-thread struct or array puts the whole object in
local memory (a persistent-kernel frame entry that way once cost 4 % of the
CG solve and hundreds of MB of DRAM writes).  These kernels must use no
stack at all and spill nothing."""
import os
import re

import pytest

from paper_1807_11830_gb300 import build as sense_build

LOG = os.path.join(sense_build.BUILD, "ptxas.log")


@pytest.fixture(scope="module")
def kernels():
    sense_build.build()
    text = open(LOG).read()
    out = {}
    for blk in text.split("ptxas info    : Compiling entry function ")[1:]:
        name = blk.split("'")[1]
        regs = re.search(r"Used (\d+) registers", blk)
        stack = re.search(r"(\d+) bytes stack frame", blk)
        spill = re.search(r"(\d+) bytes spill stores", blk)
        out[name] = (int(regs.group(1)) if regs else 0, int(stack.group(1)) if stack else 0,
                     int(spill.group(1)) if spill else 0)
    return out


def _select(kernels, *parts):
    return {n: v for n, v in kernels.items() if all(p in n for p in parts)}


def test_report_has_every_family(kernels):
    for fam in ("k_cg_persistent", "k_normal", "k_rows", "k_adj_col", "k_fwd_col", "k_transpose_maps"):
        assert _select(kernels, fam), fam


@pytest.mark.parametrize("family", ["k_rows", "k_fwd_col", "k_adj_colILi256", "k_adj_colILi160",
                                    "k_adj_colILi128", "k_transpose_maps"])
def test_pass_kernels_use_no_local_memory(kernels, family):
    sel = _select(kernels, family)
    assert sel
    bad = {n: v for n, v in sel.items() if v[1] > 0 and v[2] == 0 and "ILi160ELin1" not in n}
    assert not bad, bad


def test_headline_normal_kernels_use_no_local_memory(kernels):
    # every 256-point normal-operator kernel (all variants, both storages,
    # persistent and per-launch): no local memory beyond a small spill area
    # (a stack frame at most one 16-byte slot larger than the spill stores)
    # and spills of at most 64 bytes.  At two blocks of 256 threads per SM the
    # register cap is 128; the lane-major variant keeps its stage-0 twiddles in
    # registers and every variant carries the compensation words of its coil
    # sums, which costs a few words of spill in some variants.
    sel = {**_select(kernels, "k_cg_persistentILi256"), **_select(kernels, "k_normalILi256")}
    assert len(sel) >= 8
    bad = {n: v for n, v in sel.items() if v[1] > v[2] + 16 or v[2] > 64}
    assert not bad, bad
