"""The paper's host <-> device copy strategies (Sec. 2 "Online stage" step
(2), Table 1) through sv_copy_probe: every strategy delivers every amplitude
to its position, in both directions."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("strategy", ["sync", "async", "buffer"])
@pytest.mark.parametrize("direction", ["h2d", "d2h"])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_copy_strategies_deliver_every_amplitude(strategy, direction, dtype):
    from paper_2309_16979_gb300 import copy_probe
    sec, ok = copy_probe(14, strategy, direction, dtype, sample=4096 if strategy == "async" else 0)
    assert ok
    assert sec > 0


def test_copy_probe_rejects_bad_arguments():
    from paper_2309_16979_gb300 import copy_probe
    from paper_2309_16979_gb300._abi import SvError
    with pytest.raises(SvError):
        copy_probe(40, "sync")
