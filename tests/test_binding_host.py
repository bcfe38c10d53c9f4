"""Argument checks of the Python binding that happen on the host, before
any library call (no GPU needed)."""
import pytest
import torch

import paper_1505_04650_gb300 as cn


def test_right_factor_binding_rejects_bad_anchors():
    Rt = torch.zeros(10, 4, dtype=torch.float32)
    with pytest.raises(ValueError):
        cn.snmf_right_factor(Rt, torch.zeros(2, dtype=torch.int32))
    with pytest.raises(ValueError):
        cn.snmf_right_factor(Rt.to(torch.bfloat16), torch.zeros(2, dtype=torch.int64))
