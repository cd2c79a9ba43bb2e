"""Host logic of the output manager (§3.1 of the paper: output restricted in
time to a window and a frequency): the frame schedule, a pure function of
the library callable without a GPU."""
import pytest

from paper_1503_02464_gb300 import capi


def _req(first, last, every):
    return capi.make_output(capi.PIC_OUT_FIELD, 0, (0, 0, 0), (1, 1, 1), first, last, every)


@pytest.mark.parametrize("first,last,every", [(1, 10, 1), (3, 20, 4), (5, 5, 7), (0, 9, 3), (2, 1000, 250)])
def test_output_schedule(first, last, every):
    capi.load()
    r = _req(first, last, every)
    got = [s for s in range(0, last + 30) if capi.pic_output_due(r, s)]
    want = list(range(first, last + 1, every))
    assert got == want


def test_output_schedule_rejects_bad_period():
    capi.load()
    assert not capi.pic_output_due(_req(1, 10, 0), 1)
    assert not capi.pic_output_due(_req(1, 10, -2), 1)
