"""Host-side consistency of the index checks of the debug build (no GPU).

A kernel index outside its buffer is reported with a 16-bit tag of its source file's name; the
host maps the tag back through a table of file names.  Every source file that carries index marks
must be in that table, and the tags of the table's names must be distinct.
"""
import glob
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1806_07390_gb300", "csrc")


def file_tag(name: str) -> int:
    # FNV-1a of the base name folded to 16 bits, as fxb_file_tag computes it
    h = 2166136261
    for ch in os.path.basename(name).encode():
        h ^= ch
        h = (h * 16777619) & 0xFFFFFFFF
    return (h ^ (h >> 16)) & 0xFFFF


def host_table():
    src = open(os.path.join(CSRC, "fx_api.cu")).read()
    body = src[src.index("std::string bounds_message"):]
    body = body[:body.index("};")]
    return re.findall(r'"([\w.]+)"', body)


def test_every_marked_source_file_is_in_the_host_table():
    marked = set()
    for p in glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(CSRC, "*.h")):
        if os.path.basename(p) == "fx_check.cuh":
            continue
        if re.search(r"\bFX(I|P|PR|I_AT|P_AT)\(", open(p).read()):
            marked.add(os.path.basename(p))
    assert marked, "no marked sources found"
    assert marked <= set(host_table()), marked - set(host_table())


def test_file_tags_are_distinct_and_match_a_known_value():
    names = host_table()
    tags = [file_tag(n) for n in names]
    assert len(set(tags)) == len(tags)
    # the probe's tag as the GPU build computed it (tests/cuda/bounds_probe.cu, read back through
    # fx_probe_tag on the device toolchain's host side)
    assert file_tag("bounds_probe.cu") == 28335
