"""CPU checks of the serving SM partition: class budgets while both size
classes run, the whole GPU for a class alone, even splits with a floor."""

import pytest

from paper_2204_07816_gb300.serving import Request, _Partition


def _req(rid, L):
    return Request(rid=rid, L=L)


def test_single_class_gets_the_whole_gpu():
    p = _Partition(152)
    p.add(_req(0, 10))
    assert p.limit(0) == 0 and p.class_budget(False) == 0
    p.add(_req(1, 12))
    assert p.limit(0) == 76 and p.limit(1) == 76


def test_mixed_classes_split_the_sms():
    p = _Partition(152, large_frac=0.5)
    p.add(_req(0, 36))
    p.add(_req(1, 6))
    p.add(_req(2, 8))
    p.add(_req(3, 24))
    assert p.class_budget(True) == 76 and p.class_budget(False) == 76
    assert p.limit(0) == 38 and p.limit(3) == 38
    assert p.limit(1) == 38 and p.limit(2) == 38
    p.remove(0)
    p.remove(3)
    assert p.limit(1) == 76 and p.class_budget(False) == 0


def test_floor_and_fraction():
    p = _Partition(152, large_frac=0.25, min_sms=4)
    p.add(_req(0, 36))
    for k in range(1, 60):
        p.add(_req(k, 6))
    assert p.class_budget(True) == 38 and p.class_budget(False) == 114
    assert p.limit(0) == 38
    assert p.limit(5) == 4          # 114 // 59 = 1, raised to the floor
