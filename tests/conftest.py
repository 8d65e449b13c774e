import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")


@pytest.fixture(scope="session")
def mech_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("mechs"))


@pytest.fixture(scope="session")
def mech_path(mech_dir):
    from paper_2205_05681_gb300 import synth

    def get(name):
        return synth.mechanism_file(name, mech_dir)

    return get


@pytest.fixture(scope="session")
def omech(mech_path):
    """Oracle-side mechanisms, parsed once per session."""
    from oracle import oracle as O
    cache = {}

    def get(name):
        if name not in cache:
            path = os.path.join(GOLDEN, name) if name.endswith(".mech") else mech_path(name)
            cache[name] = O.Mechanism(path)
        return cache[name]

    return get


def states(name, n, recipe, seed):
    from paper_2205_05681_gb300 import synth
    return synth.make_states(synth.mechanism(name), n, recipe, seed)


def shuffled_spec(src, dst, seed):
    """Copy a mechanism spec with its reactions (each R line with its EFF/LOW/TROE lines) in a
    seeded random order; returns perm with new reaction i = old reaction perm[i]."""
    lines = open(src).read().splitlines()
    head = []
    blocks = []
    tail = []
    i = 0
    while not lines[i].startswith("REACTIONS"):
        head.append(lines[i])
        i += 1
    head.append(lines[i])
    i += 1
    while i < len(lines) and not lines[i].startswith("END"):
        if lines[i].startswith("R "):
            blocks.append([lines[i]])
        elif lines[i].strip() and not lines[i].startswith("#"):
            blocks[-1].append(lines[i])
        i += 1
    tail = lines[i:]
    perm = np.random.default_rng(seed).permutation(len(blocks))
    with open(dst, "w") as fh:
        fh.write("\n".join(head + [l for p in perm for l in blocks[p]] + tail) + "\n")
    return perm
