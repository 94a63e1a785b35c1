"""The seeded generators give the same graphs on every host: the SHA-256 of
each workload's inputs equals the value stored with the oracle's results."""
from __future__ import annotations

import hashlib

from gen import configs
from gpu_common import golden


def test_er1000_inputs():
    g = golden("er1000")
    w = configs.er1000()
    assert w.targets[0].sha256() == g["target_sha256"] and w.patterns[0].sha256() == g["pattern_sha256"]


def test_er2000_inputs():
    g = golden("er2000")
    w = configs.er2000()
    assert w.targets[0].sha256() == g["target_sha256"]
    assert [p.sha256() for p in w.patterns] == [e["pattern_sha256"] for e in g["patterns"]]


def test_cl10k_inputs():
    g = golden("cl10k")
    w = configs.cl10k()
    assert w.targets[0].sha256() == g["target_sha256"]
    assert [p.sha256() for p in w.patterns] == [e["pattern_sha256"] for e in g["patterns"]]


def test_mol200_inputs():
    g = golden("mol200")
    ts = configs.mol_targets(200)
    ps = configs.mol_patterns(ts, 1000)
    h = hashlib.sha256()
    for x in ts + ps:
        h.update(x.sha256().encode())
    assert h.hexdigest() == g["inputs_sha256"]


def test_cl100k_target():
    assert configs.cl100k_target().sha256() == golden("cl100k")["target_sha256"]
