"""Host-side checks of the C ABI library that need no GPU: it builds, loads, exports every
declared symbol, and its host CBC construction matches the oracle's."""
import os
import re

import numpy as np
import pytest

from oracle import lattice
from paper_2103_03407_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mlqmc_evp.h")).read()
    return sorted(set(re.findall(r"^(?:mq_status|const char\*)\s+(mq_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(binding.EXPORTS)


@pytest.mark.parametrize("N,s", [(8, 3), (64, 6), (256, 16), (1024, 8)])
def test_cbc_matches_oracle(lib, N, s):
    # integer output: bit-exact
    assert np.array_equal(binding.mq_cbc_lattice(N, s), lattice.cbc(N, s))


@pytest.mark.parametrize("m_min,m_max,s", [(1, 4, 4), (3, 7, 6), (5, 5, 5), (6, 9, 12)])
def test_embedded_cbc_matches_oracle(lib, m_min, m_max, s):
    assert np.array_equal(binding.mq_cbc_embedded_lattice(m_min, m_max, s), lattice.embedded_cbc(m_min, m_max, s))


def test_cbc_rejects_bad_arguments(lib):
    with pytest.raises(binding.MQError):
        binding.mq_cbc_embedded_lattice(4, 3, 2)
    with pytest.raises(binding.MQError):
        binding.mq_cbc_lattice(1, 3)


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.MQError):
        binding.Context(0)
