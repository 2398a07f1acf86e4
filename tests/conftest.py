import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def I():
    from paper_2306_11006_gb300 import inputs
    return inputs


class Keys:
    def __init__(self, O, I, seed, n, **kw):
        self.n = n
        self.kr = I.key_randomness(seed, n, **kw)
        self.bsk, self.ksk = O.keygen(self.kr)
        self.ctx = O.Context(n, self.bsk, self.ksk)
        self.s = self.kr.s
        self.K = self.kr.K

    def encrypt(self, O, I, bits, seed):
        m, e = I.encryption_randomness(seed, len(bits), self.n)
        return O.encrypt(self.n, self.s, m, e, np.asarray(bits, np.uint8))


@pytest.fixture(scope="session")
def keys630(O, I):
    return Keys(O, I, 0, 630)


@pytest.fixture(scope="session")
def keys64(O, I):
    return Keys(O, I, 5, 64)


@pytest.fixture(scope="session")
def keys512_l2(O, I):
    """The paper's own parameter set: n = 512, gadget l = 2 (Bg = 2^10)."""
    return Keys(O, I, 7, 512, l=2)
