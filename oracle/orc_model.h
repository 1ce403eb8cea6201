/*
 * Model parameters shared by the oracle's translation units (phd_oracle.c,
 * birth_oracle.c).  TEST INFRASTRUCTURE ONLY; not used by the CUDA path.
 */
#ifndef ORC_MODEL_H
#define ORC_MODEL_H

#define ORC_LINEAR 0
#define ORC_RANGE_BEARING 1
#define ORC_BIRTH_UNIFORM 0
#define ORC_BIRTH_GAUSSIAN 1

typedef struct {
    int meas_model;       /* ORC_LINEAR or ORC_RANGE_BEARING */
    int birth_model;      /* ORC_BIRTH_UNIFORM or ORC_BIRTH_GAUSSIAN */
    double dt;            /* sampling period T (Sec. 4: T = 1) */
    double sigma_a;       /* std of the acceleration noise w_k */
    double sigma_z[2];    /* linear: (sx, sy) m; range-bearing: (sr m, stheta rad) */
    double sensor[2];     /* sensor position (s_x, s_y) */
    double region[4];     /* x_min, x_max, y_min, y_max */
    double r_max;         /* range-bearing clutter support: r in [0, r_max] */
    double p_s;           /* survival probability e_{k|k-1} */
    double p_d;           /* detection probability P_D */
    double clutter_rate;  /* lambda_k: mean clutter count per scan */
    double birth_mass;    /* nu_b: expected number of births per step */
    double birth_vel_sigma;
    double sigma_a_y;     /* acceleration noise std of the y axis (0: sigma_a) */
    double theta_span;    /* range-bearing clutter bearing extent (0: 2 pi) */
    double birth_mean[4]; /* Gaussian birth N(x_bar, Q) of Sec. 4: mean [x, vx, y, vy] */
    double birth_std[4];  /* and the square roots of Q's diagonal */
    double gate_sigma;    /* > 0: g truncated to 0 at Mahalanobis distance >= gate_sigma */
} orc_model;

#endif /* ORC_MODEL_H */
