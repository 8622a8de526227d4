// p_add against the QBX order p = 0..16, measured by calibrate_p_add.py
// (the experiment of Sec. 7.1: 50 random curves r = 5 + sum_j delta_j sin jt,
// k = 5, Green's identity at targets near the boundary, seed 2016): the
// non-decreasing envelope of the largest p' found per calibrated p; orders
// between calibrated ones take the value of the next calibrated order.
// Generated file: rerun the script instead of editing it.
#pragma once
constexpr int kPAddCalibrated[17] = {0, 0, 0, 3, 3, 7, 7, 9, 9, 9, 9, 10, 10, 11, 11, 11, 11};
