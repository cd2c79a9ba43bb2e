"""bench.py host helpers that need no GPU: the sysfs CPU-list parser and the
PCI bus-id mapping used to place the end-to-end input buffers near the GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_parse_cpulist():
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()


def test_pci_sysfs_name():
    assert bench.pci_sysfs_name("00000009:01:00.0\n") == "0009:01:00.0"
    assert bench.pci_sysfs_name("0000:1B:00.0") == "0000:1b:00.0"
