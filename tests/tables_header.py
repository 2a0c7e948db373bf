"""Reads the constant tables of the CUDA library's generated header as text."""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2508_08965_gb300", "csrc", "cgks_tables.h")


def read_table(name):
    txt = open(HDR).read()
    m = re.search(r"(?:CGKS_G?TABLE double|static const int) %s((?:\[\d+\])+) = \{(.*?)\};" % re.escape(name),
                  txt, re.S)
    if not m:
        raise KeyError(name)
    shape = [int(x) for x in re.findall(r"\[(\d+)\]", m.group(1))]
    nums = re.findall(r"[-+]?\d+\.?\d*(?:[eE][-+]?\d+)?", m.group(2))
    return np.array([float(x) for x in nums]).reshape(shape)
