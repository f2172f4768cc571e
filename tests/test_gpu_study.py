"""The paper's protocol (section IV) at L = 16 on ten synthetic coupling sets:
the improved exchanges raise the acceptance and shorten the round-trip time
as Tables I and II report (decimation ~2.1x, cooling/heating ~2.4-2.6x).
Trends only: the paper's coupling sets are not available."""
import json

import pytest

from paper_1006_4247_gb300 import study

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


def test_paper_protocol_trends_L16():
    out = study.protocol(16, 15, n_sets=10, cycles=10000, burn=2000)
    print("\npaper protocol, L = 16:", json.dumps({m: {k: v[k] for k in v if not k.endswith("per_set")}
                                                  for m, v in out["methods"].items()}))
    ms = out["methods"]
    # Table I: standard acceptance about 0.11-0.13 over the ladder
    assert 0.09 < ms["plain"]["acc_first_pair"][0] and ms["plain"]["acc_last_pair"][1] < 0.15
    # Table II: acceptance and round-trip speed-ups
    assert 1.85 < ms["decimation"]["acc_ratio"] < 2.35
    assert 2.1 < ms["coolheat"]["acc_ratio"] < 2.9
    assert ms["decimation"]["t_R_speedup_mean"] > 1.7
    assert ms["coolheat"]["t_R_speedup_mean"] > 2.0
    assert ms["decimation"]["tau_speedup_median"] > 1.5
