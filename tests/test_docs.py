"""The documents point at files that exist, and every profile summary gives
the ncu command that produced it (with --clock-control none)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2311_14616_gb300")


def _paths(doc):
    text = open(os.path.join(ROOT, doc)).read()
    for m in re.finditer(r"`([A-Za-z0-9_./-]+\.(?:cu|cuh|py|h|c|md|json))`", text):
        p = m.group(1)
        if p.endswith(("BASELINE.json", "MEASURED_PEAKS.json")):
            continue          # written by the environment, not by this repository
        yield p


def _exists(p):
    cands = [os.path.join(ROOT, p), os.path.join(PKG, p)]
    return any(os.path.exists(c) for c in cands)


@pytest.mark.parametrize("doc", ["DESIGN.md", "README.md"])
def test_documents_name_existing_files(doc):
    missing = sorted({p for p in _paths(doc) if "/" in p and not _exists(p)})
    assert not missing, missing


def test_profiles_give_their_command():
    prof = os.path.join(ROOT, "profiles")
    files = [f for f in os.listdir(prof) if f.endswith((".md", ".txt"))]
    assert files
    for f in files:
        text = open(os.path.join(prof, f)).read()
        assert re.search(r"^\s*ncu .*--clock-control none", text, re.M), f
        assert "gpurun" not in text and "/root/" not in text, f
