"""Host logic of the measurement drivers that needs no GPU."""

import pytest

from paper_2108_07031_gb300 import lskum as L
from paper_2108_07031_gb300.precision_study import parse_options


def test_precision_study_option_parsing():
    opts = parse_options(["wall_factor=1.0", "order=1", "weight_power=2e0", "outer_mode=0"])
    assert opts == {"wall_factor": 1.0, "order": 1, "weight_power": 2.0, "outer_mode": 0}
    assert isinstance(opts["order"], int) and isinstance(opts["wall_factor"], float)
    # every name is a field of the library's options struct
    o = L.Options()
    for name in opts:
        assert hasattr(o, name)
    for bad in ("order", "=1", "order:1"):
        with pytest.raises(ValueError):
            parse_options([bad])
